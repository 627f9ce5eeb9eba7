// Batched, uneven multi-mesh tracing: one persistent launch walks the rays
// of many meshes from a single global work queue (a device descriptor table
// per mesh; each lane finds its mesh by binary search over the meshes' first
// ray index), optionally after sorting every chunk of G rays by start
// location and direction octant.  The sort and the trace are captured once
// in a CUDA graph and replayed.  An autotuner picks block size, refill
// threshold, steps between refills and the sort chunk by timing them.
#include <algorithm>
#include <cstring>
#include <vector>

#include "tm_internal.h"

struct tm_batch {
    std::vector<const tm_mesh *> meshes;
    std::vector<BatchDesc> descs;
    BatchDesc *d_descs = nullptr;
    std::vector<int32_t *> perm;
    std::vector<int64_t> perm_cap;
    int4 *d_chunks = nullptr;  // (mesh, first ray, count, 0) per sort chunk
    int64_t n_chunks = 0, chunks_cap = 0;
    unsigned long long *d_cursor = nullptr;  // walk scratch (counters + parked list)
    size_t cursor_bytes = 0;
    TraceConfig cfg{};
    int32_t sort_chunk = 0;
    int64_t total = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int graph_kernels = 0;
};

namespace tmk {

constexpr int kMaxSortChunk = 4096;

__global__ void __launch_bounds__(1024)
sort_chunks_kernel(const BatchDesc *__restrict__ descs, const int4 *__restrict__ chunks) {
    __shared__ unsigned long long s[kMaxSortChunk];
    const int4 ch = chunks[blockIdx.x];
    const BatchDesc &D = descs[ch.x];
    const int len = ch.z;
    int P = 1;
    while (P < len) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        unsigned long long v = ~0ull;
        if (i < len) {
            const float4 w0 = __ldg(reinterpret_cast<const float4 *>(D.rays + ch.y + i));
            const float4 w1 = __ldg(reinterpret_cast<const float4 *>(D.rays + ch.y + i) + 1);
            const int32_t st = __float_as_int(w0.w);
            uint32_t where;
            if (st >= 0) {
                where = (uint32_t)st >> 6;                    // Hilbert-ordered tet ids: nearby tets
            } else {
                const int32_t c = (-1 - st) >> 1;
                where = (uint32_t)__ldg(&D.mesh.cface[2 * c].y) >> 6;
            }
            const uint32_t oct = (w1.x < 0.f) | ((w1.y < 0.f) << 1) | ((w1.z < 0.f) << 2);
            const uint32_t key = ((where & 0x0FFFFFFFu) << 3) | oct;    // place, then direction class
            v = ((unsigned long long)key << 32) | (unsigned)i;
        }
        s[i] = v;
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int x = i ^ j;
                if (x > i) {
                    const bool up = (i & k) == 0;
                    const unsigned long long a = s[i], b = s[x];
                    if ((a > b) == up) {
                        s[i] = b;
                        s[x] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    int32_t *perm = const_cast<int32_t *>(D.perm);
    for (int i = threadIdx.x; i < len; i += blockDim.x)
        perm[ch.y + i] = ch.y + (int32_t)(s[i] & 0xffffffffu);
}

}  // namespace tmk

namespace {

void destroy_graph(tm_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

tm_status build_graph(tm_batch *b) {
    destroy_graph(b);
    if (!b->cap_stream) TM_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
    TM_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
    tm_status st = TM_OK;
    int kernels = 0;
    if (b->sort_chunk > 0 && b->n_chunks > 0) {
        tmk::sort_chunks_kernel<<<(unsigned)b->n_chunks, 1024, 0, b->cap_stream>>>(b->d_descs, b->d_chunks);
        ++kernels;
    }
    st = launch_trace_batch(b->d_descs, (int)b->meshes.size(), b->total, b->cfg, b->d_cursor,
                            b->cap_stream, false);
    if (b->total > 0) kernels += 3;  // start, walk, finish
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
    if (st != TM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) {
        tm_set_error("cudaStreamEndCapture", e);
        return TM_ERR_CUDA;
    }
    e = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        tm_set_error("cudaGraphInstantiate", e);
        return TM_ERR_CUDA;
    }
    b->graph_kernels = kernels;
    return TM_OK;
}

}  // namespace

extern "C" {

tm_status tm_batch_create(const tm_mesh *const *meshes, int n_meshes, tm_batch **out) {
    if (!out || !meshes || n_meshes < 1 || n_meshes > 64) return TM_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n_meshes; ++i) {
        if (!meshes[i]) return TM_ERR_ARG;
        if (!meshes[i]->on_device) return TM_ERR_NO_DEVICE;
    }
    tm_batch *b = new tm_batch();
    b->meshes.assign(meshes, meshes + n_meshes);
    b->descs.resize((size_t)n_meshes);
    b->perm.assign((size_t)n_meshes, nullptr);
    b->perm_cap.assign((size_t)n_meshes, 0);
    cudaError_t e;
    if ((e = cudaMalloc(&b->d_descs, sizeof(BatchDesc) * (size_t)n_meshes)) != cudaSuccess ||
        (e = cudaMalloc(&b->d_cursor, batch_scratch_bytes(0))) != cudaSuccess) {
        tm_set_error("cudaMalloc", e);
        tm_batch_destroy(b);
        return TM_ERR_CUDA;
    }
    b->cursor_bytes = batch_scratch_bytes(0);
    b->cfg = resolve_trace_opts(nullptr, 1);
    *out = b;
    return TM_OK;
}

tm_status tm_batch_set(tm_batch *b, const tm_ray *const *rays, const int64_t *n, tm_hit *const *hits,
                       const tm_trace_opts *opts, int32_t sort_chunk) {
    if (!b || !rays || !n || !hits) return TM_ERR_ARG;
    if (sort_chunk < 0 || sort_chunk > tmk::kMaxSortChunk) return TM_ERR_ARG;
    const int nm = (int)b->meshes.size();
    int64_t max_nt = 1, offset = 0;
    std::vector<int4> chunks;
    for (int i = 0; i < nm; ++i) {
        if (n[i] < 0 || (n[i] > 0 && (!rays[i] || !hits[i]))) return TM_ERR_ARG;
        if ((((uintptr_t)rays[i]) | ((uintptr_t)hits[i])) & 31u) return TM_ERR_ARG;
        if (n[i] > INT32_MAX) return TM_ERR_TOO_LARGE;
        max_nt = std::max<int64_t>(max_nt, b->meshes[(size_t)i]->nt);
        BatchDesc &D = b->descs[(size_t)i];
        D.mesh = mesh_view(b->meshes[(size_t)i]);
        D.rays = rays[i];
        D.hits = hits[i];
        D.n = n[i];
        D.offset = offset;
        D.perm = nullptr;
        if (sort_chunk > 0 && n[i] > 0) {
            if (b->perm_cap[(size_t)i] < n[i]) {
                cudaFree(b->perm[(size_t)i]);
                b->perm[(size_t)i] = nullptr;
                TM_CUDA(cudaMalloc(&b->perm[(size_t)i], sizeof(int32_t) * (size_t)n[i]));
                b->perm_cap[(size_t)i] = n[i];
            }
            D.perm = b->perm[(size_t)i];
            for (int64_t s = 0; s < n[i]; s += sort_chunk)
                chunks.push_back(make_int4(i, (int)s, (int)std::min<int64_t>(sort_chunk, n[i] - s), 0));
        }
        offset += n[i];
    }
    b->total = offset;
    if (batch_scratch_bytes(offset) > b->cursor_bytes) {
        cudaFree(b->d_cursor);
        b->d_cursor = nullptr;
        TM_CUDA(cudaMalloc(&b->d_cursor, batch_scratch_bytes(offset)));
        b->cursor_bytes = batch_scratch_bytes(offset);
    }
    b->cfg = resolve_trace_opts(opts, max_nt);
    if (b->cfg.format == TM_FORMAT_AUTO) {
        bool all_faces = true, all_faces16 = true;
        for (const tm_mesh *m : b->meshes) {
            all_faces = all_faces && m->d_face;
            all_faces16 = all_faces16 && m->d_face16;
        }
        b->cfg.format = auto_format(all_faces16, all_faces);
    }
    if (b->cfg.format == TM_FORMAT_TET20) return TM_ERR_ARG;  // two arrays per mesh: not batched
    for (const tm_mesh *m : b->meshes) {
        if (b->cfg.format == TM_FORMAT_TET20_AOS && !m->d_t20aos) return TM_ERR_ARG;
        if (b->cfg.format == TM_FORMAT_FACE && !m->d_face) return TM_ERR_ARG;
        if (b->cfg.format == TM_FORMAT_FACE16 && !m->d_face16) return TM_ERR_ARG;
    }
    b->sort_chunk = sort_chunk;
    b->n_chunks = (int64_t)chunks.size();
    if (b->n_chunks > b->chunks_cap) {
        cudaFree(b->d_chunks);
        b->d_chunks = nullptr;
        TM_CUDA(cudaMalloc(&b->d_chunks, sizeof(int4) * (size_t)b->n_chunks));
        b->chunks_cap = b->n_chunks;
    }
    if (b->n_chunks)
        TM_CUDA(cudaMemcpy(b->d_chunks, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice));
    TM_CUDA(cudaMemcpy(b->d_descs, b->descs.data(), sizeof(BatchDesc) * (size_t)nm, cudaMemcpyHostToDevice));
    return build_graph(b);
}

tm_status tm_batch_run(tm_batch *b, void *stream) {
    if (!b || !b->exec) return TM_ERR_ARG;
    TM_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    tm_count_launches((uint64_t)b->graph_kernels);
    return TM_OK;
}

tm_status tm_batch_run_separate(tm_batch *b, void *stream) {
    if (!b) return TM_ERR_ARG;
    for (size_t i = 0; i < b->meshes.size(); ++i) {
        const BatchDesc &D = b->descs[i];
        const tm_status st = launch_trace(D.mesh, D.rays, D.n, nullptr, D.hits, b->cfg, (cudaStream_t)stream);
        if (st != TM_OK) return st;
    }
    return TM_OK;
}

tm_status tm_batch_autotune(tm_batch *b, int reps, tm_tuned *best, void *stream) {
    if (!b || reps < 1) return TM_ERR_ARG;
    const int nm = (int)b->meshes.size();
    std::vector<const tm_ray *> rays((size_t)nm);
    std::vector<tm_hit *> hits((size_t)nm);
    std::vector<int64_t> n((size_t)nm);
    for (int i = 0; i < nm; ++i) {
        rays[(size_t)i] = b->descs[(size_t)i].rays;
        hits[(size_t)i] = b->descs[(size_t)i].hits;
        n[(size_t)i] = b->descs[(size_t)i].n;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    TM_CUDA(cudaEventCreate(&e0));
    TM_CUDA(cudaEventCreate(&e1));
    tm_trace_opts o{};
    o.mode = b->cfg.mode;
    o.guard_tau = b->cfg.tau;
    o.max_steps = b->cfg.max_steps;
    o.block = b->cfg.block;
    o.refill = b->cfg.refill;
    o.batch_steps = b->cfg.batch_steps;
    o.format = b->cfg.format;
    int32_t chunk = b->sort_chunk;
    auto measure = [&](const tm_trace_opts &opt, int32_t sc, float *ms) -> tm_status {
        tm_status st = tm_batch_set(b, rays.data(), n.data(), hits.data(), &opt, sc);
        if (st != TM_OK) return st;
        if ((st = tm_batch_run(b, stream)) != TM_OK) return st;  // warm-up
        TM_CUDA(cudaEventRecord(e0, s));
        for (int r = 0; r < reps; ++r)
            if ((st = tm_batch_run(b, stream)) != TM_OK) return st;
        TM_CUDA(cudaEventRecord(e1, s));
        TM_CUDA(cudaEventSynchronize(e1));
        TM_CUDA(cudaEventElapsedTime(ms, e0, e1));
        *ms /= (float)reps;
        return TM_OK;
    };
    float best_ms = 0.f;
    tm_status st = measure(o, chunk, &best_ms);
    const int blocks[] = {128, 256, 384, 512, 576};
    const int refills[] = {4, 8, 16, 24, 32};
    const int steps[] = {2, 4, 8, 16, 32};
    const int chunks[] = {0, 256, 1024, 4096};
    bool all_faces = true, all_faces16 = true;
    for (const tm_mesh *m : b->meshes) {
        all_faces = all_faces && m->d_face;
        all_faces16 = all_faces16 && m->d_face16;
    }
    const int formats[] = {auto_format(all_faces16, all_faces), TM_FORMAT_TET32, TM_FORMAT_TET16};
    for (int pass = 0; pass < 2 && st == TM_OK; ++pass) {
        for (int v : formats) {
            tm_trace_opts c = o; c.format = v; float ms;
            if ((st = measure(c, chunk, &ms)) != TM_OK) break;
            if (ms < best_ms) { best_ms = ms; o = c; }
        }
        for (int v : blocks) {
            if (st != TM_OK) break;
            tm_trace_opts c = o; c.block = v; float ms;
            if ((st = measure(c, chunk, &ms)) != TM_OK) break;
            if (ms < best_ms) { best_ms = ms; o = c; }
        }
        for (int v : refills) {
            if (st != TM_OK) break;
            tm_trace_opts c = o; c.refill = v; float ms;
            if ((st = measure(c, chunk, &ms)) != TM_OK) break;
            if (ms < best_ms) { best_ms = ms; o = c; }
        }
        for (int v : steps) {
            if (st != TM_OK) break;
            tm_trace_opts c = o; c.batch_steps = v; float ms;
            if ((st = measure(c, chunk, &ms)) != TM_OK) break;
            if (ms < best_ms) { best_ms = ms; o = c; }
        }
        for (int v : chunks) {
            if (st != TM_OK) break;
            float ms;
            if ((st = measure(o, v, &ms)) != TM_OK) break;
            if (ms < best_ms) { best_ms = ms; chunk = v; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != TM_OK) return st;
    st = tm_batch_set(b, rays.data(), n.data(), hits.data(), &o, chunk);
    if (best) {
        best->opts = o;
        best->sort_chunk = chunk;
        best->ms = best_ms;
    }
    return st;
}

void tm_batch_destroy(tm_batch *b) {
    if (!b) return;
    destroy_graph(b);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int32_t *p : b->perm) cudaFree(p);
    cudaFree(b->d_chunks);
    cudaFree(b->d_descs);
    cudaFree(b->d_cursor);
    delete b;
}

}  // extern "C"
