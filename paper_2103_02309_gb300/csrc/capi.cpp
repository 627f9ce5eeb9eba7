// The extern "C" entry points declared in include/tetmesh.h: argument
// checks, option defaults, and calls into the host build and the launchers.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "tm_internal.h"

tm_status tm_build_host(const float *points, int64_t np, const int32_t *tets, int64_t nt,
                        const int32_t *tris, int64_t nc, const tm_build_opts *opts, tm_mesh *m);
tm_status tm_upload(tm_mesh *m);
void tm_free_device(tm_mesh *m);
uint64_t tm_hilbert3(uint32_t x, uint32_t y, uint32_t z, int bits);

namespace {
thread_local std::string g_error;
std::atomic<uint64_t> g_launches{0};
}  // namespace

void tm_set_error(const char *what, cudaError_t e) {
    g_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
}
void tm_set_error_text(const std::string &s) { g_error = s; }
void tm_count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

extern "C" {

const char *tm_status_str(tm_status s) {
    switch (s) {
        case TM_OK: return "ok";
        case TM_ERR_ARG: return "invalid argument";
        case TM_ERR_RANGE: return "vertex id out of range";
        case TM_ERR_ORIENT: return "tet with non-positive orientation";
        case TM_ERR_NONMANIFOLD: return "face shared by more than two tets";
        case TM_ERR_CFACE_UNMATCHED: return "constrained triangle is not a tet face";
        case TM_ERR_CFACE_DUPLICATE: return "two constrained triangles on one tet face";
        case TM_ERR_OOM: return "out of memory";
        case TM_ERR_CUDA: return "CUDA error";
        case TM_ERR_TOO_LARGE: return "mesh or ray batch too large";
        case TM_ERR_NO_DEVICE: return "mesh has no device copy";
    }
    return "unknown status";
}

const char *tm_last_error(void) { return g_error.c_str(); }

uint64_t tm_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

tm_status tm_build(const float *points, int64_t n_points, const int32_t *tets, int64_t n_tets,
                   const int32_t *tris, int64_t n_tris, const tm_build_opts *opts, int upload,
                   tm_mesh **out) {
    if (!out) return TM_ERR_ARG;
    *out = nullptr;
    if (!points || !tets || n_points <= 0 || n_tets <= 0 || n_tris < 0 || (n_tris > 0 && !tris))
        return TM_ERR_ARG;
    if (n_points > INT32_MAX || n_tets > INT32_MAX || n_tris >= (int64_t(1) << 30))
        return TM_ERR_TOO_LARGE;
    tm_mesh *m = new (std::nothrow) tm_mesh();
    if (!m) return TM_ERR_OOM;
    tm_status st;
    try {
        st = tm_build_host(points, n_points, tets, n_tets, tris, n_tris, opts, m);
    } catch (const std::bad_alloc &) {
        st = TM_ERR_OOM;
    }
    if (st == TM_OK && upload) st = tm_upload(m);
    if (st != TM_OK) {
        tm_free_device(m);
        delete m;
        return st;
    }
    *out = m;
    return TM_OK;
}

void tm_destroy(tm_mesh *mesh) {
    if (!mesh) return;
    tm_free_device(mesh);
    delete mesh;
}

tm_status tm_mesh_info_get(const tm_mesh *m, tm_mesh_info *info) {
    if (!m || !info) return TM_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    info->n_points = m->np;
    info->n_tets = m->nt;
    info->n_tris = m->nc;
    info->extent = m->extent;
    for (int a = 0; a < 3; ++a) {
        info->bbox_lo[a] = m->lo[a];
        info->bbox_hi[a] = m->hi[a];
    }
    info->source_tet = m->source_tet;
    info->on_device = m->on_device ? 1 : 0;
    info->tet16_dev = m->d_tet16;
    info->points_dev = m->d_pts;
    info->cold_dev = m->d_cold;
    info->cface_dev = m->d_cface;
    info->tet20_dev = m->d_t20;
    info->tet20_n3_dev = m->d_t20n3;
    info->tet20_aos_dev = m->d_t20aos;
    info->face_dev = m->d_face;
    info->face16_dev = m->d_face16;
    info->device_bytes = m->device_bytes;
    info->n_regions = m->n_regions;
    return TM_OK;
}

tm_status tm_mesh_export(const tm_mesh *m, int32_t *tet16, int32_t *cold, float *points,
                         int32_t *cface, int32_t *point_perm, int32_t *tet_perm) {
    if (!m) return TM_ERR_ARG;
    if (tet16) std::memcpy(tet16, m->tet16.data(), sizeof(int32_t) * m->tet16.size());
    if (cold) std::memcpy(cold, m->cold.data(), sizeof(int32_t) * m->cold.size());
    if (points) std::memcpy(points, m->pts4.data(), sizeof(float) * m->pts4.size());
    if (cface && !m->cface.empty()) std::memcpy(cface, m->cface.data(), sizeof(int32_t) * m->cface.size());
    if (point_perm) std::memcpy(point_perm, m->pperm.data(), sizeof(int32_t) * m->pperm.size());
    if (tet_perm) std::memcpy(tet_perm, m->tperm.data(), sizeof(int32_t) * m->tperm.size());
    return TM_OK;
}

tm_status tm_mesh_export_tet20(const tm_mesh *m, int32_t *vxn, int32_t *n3, int32_t *aos) {
    if (!m || m->t20.empty()) return TM_ERR_ARG;
    if (vxn) std::memcpy(vxn, m->t20.data(), sizeof(int32_t) * m->t20.size());
    if (n3) std::memcpy(n3, m->t20n3.data(), sizeof(int32_t) * m->t20n3.size());
    if (aos) std::memcpy(aos, m->t20aos.data(), sizeof(int32_t) * m->t20aos.size());
    return TM_OK;
}

tm_status tm_mesh_export_faces(const tm_mesh *m, int32_t *faces) {
    if (!m || m->face.empty() || !faces) return TM_ERR_ARG;
    std::memcpy(faces, m->face.data(), sizeof(int32_t) * m->face.size());
    return TM_OK;
}

tm_status tm_mesh_export_faces16(const tm_mesh *m, int32_t *faces16) {
    if (!m || m->face16.empty() || !faces16) return TM_ERR_ARG;
    std::memcpy(faces16, m->face16.data(), sizeof(int32_t) * m->face16.size());
    return TM_OK;
}

tm_status tm_mesh_export_restart(const tm_mesh *m, int32_t *restart) {
    if (!m || !restart) return TM_ERR_ARG;
    std::memcpy(restart, m->restart.data(), sizeof(int32_t) * m->restart.size());
    return TM_OK;
}

tm_status tm_map_ids(const tm_mesh *m, int kind, int direction, const int32_t *in, int32_t *out,
                     int64_t n) {
    if (!m || (n > 0 && (!in || !out)) || n < 0) return TM_ERR_ARG;
    const std::vector<int32_t> *map;
    if (kind == TM_IDS_TET) map = direction == TM_TO_INPUT ? &m->tperm : &m->tinv;
    else if (kind == TM_IDS_POINT) map = direction == TM_TO_INPUT ? &m->pperm : &m->pinv;
    else return TM_ERR_ARG;
    if (direction != TM_TO_INPUT && direction != TM_TO_INTERNAL) return TM_ERR_ARG;
    const int64_t sz = (int64_t)map->size();
    for (int64_t i = 0; i < n; ++i) out[i] = (in[i] >= 0 && in[i] < sz) ? (*map)[(size_t)in[i]] : -1;
    return TM_OK;
}

tm_status tm_hilbert_keys(const uint32_t *ijk, int64_t n, int bits, uint64_t *keys) {
    if ((n > 0 && (!ijk || !keys)) || n < 0 || bits < 1 || bits > 21) return TM_ERR_ARG;
    for (int64_t i = 0; i < n; ++i) keys[i] = tm_hilbert3(ijk[3 * i], ijk[3 * i + 1], ijk[3 * i + 2], bits);
    return TM_OK;
}

tm_status tm_locate(const tm_mesh *m, const float *q, int64_t n, const int32_t *hint, int32_t source,
                    int32_t *tet_out, void *stream) {
    if (!m || n < 0 || (n > 0 && (!q || !tet_out))) return TM_ERR_ARG;
    if (!m->on_device) return TM_ERR_NO_DEVICE;
    MeshView mv = mesh_view(m);
    if (source >= 0 && source < m->nt) mv.seeds = nullptr;  // an explicit source overrides the lattice
    else source = m->source_tet;
    const uint32_t bound = (uint32_t)(64.0 * std::cbrt((double)m->nt) * 8.0 + 1024.0);
    return launch_locate(mv, q, n, hint, source, tet_out, bound, (cudaStream_t)stream);
}

tm_status tm_trace(const tm_mesh *m, const tm_ray *rays, int64_t n, const int64_t *n_dev,
                   tm_hit *hits, const tm_trace_opts *opts, void *stream) {
    if (!m || n < 0 || (n > 0 && (!rays || !hits))) return TM_ERR_ARG;
    if ((((uintptr_t)rays) | ((uintptr_t)hits)) & 31u) return TM_ERR_ARG;
    if (!m->on_device) return TM_ERR_NO_DEVICE;
    const TraceConfig cfg = resolve_trace_opts(opts, m->nt);
    if (cfg.format == TM_FORMAT_TET20 && !m->d_t20) return TM_ERR_ARG;
    if (cfg.format == TM_FORMAT_TET20_AOS && !m->d_t20aos) return TM_ERR_ARG;
    if (cfg.format == TM_FORMAT_FACE && !m->d_face) return TM_ERR_ARG;
    if (cfg.format == TM_FORMAT_FACE16 && !m->d_face16) return TM_ERR_ARG;
    return launch_trace(mesh_view(m), rays, n, n_dev, hits, cfg, (cudaStream_t)stream);
}

tm_status tm_trace_shadow(const tm_mesh *m, const tm_ray *rays, int64_t n, const int64_t *n_dev,
                          const int32_t *light_tet_dev, tm_hit *hits, const tm_trace_opts *opts,
                          void *stream) {
    if (!m || n < 0 || !light_tet_dev || (n > 0 && (!rays || !hits))) return TM_ERR_ARG;
    if ((((uintptr_t)rays) | ((uintptr_t)hits)) & 31u) return TM_ERR_ARG;
    if (!m->on_device) return TM_ERR_NO_DEVICE;
    TraceConfig cfg = resolve_trace_opts(opts, m->nt);
    if (cfg.format == TM_FORMAT_TET20 && !m->d_t20) return TM_ERR_ARG;
    if (cfg.format == TM_FORMAT_TET20_AOS && !m->d_t20aos) return TM_ERR_ARG;
    if (cfg.format == TM_FORMAT_FACE && !m->d_face) return TM_ERR_ARG;
    if (cfg.format == TM_FORMAT_FACE16 && !m->d_face16) return TM_ERR_ARG;
    cfg.bounded = true;
    cfg.stop_tet = light_tet_dev;
    return launch_trace(mesh_view(m), rays, n, n_dev, hits, cfg, (cudaStream_t)stream);
}

tm_status tm_gen_primary(const tm_camera *cam, const int32_t *start_dev, float tmax, tm_ray *rays,
                         void *stream) {
    if (!cam || !start_dev || !rays || cam->width < 0 || cam->height < 0) return TM_ERR_ARG;
    if (((uintptr_t)rays) & 31u) return TM_ERR_ARG;
    return launch_gen_primary(cam, start_dev, tmax, rays, (cudaStream_t)stream);
}

tm_status tm_gen_secondary(const tm_mesh *m, const tm_hit *hits, int64_t n, const int64_t *n_dev,
                           int per_hit, float tmax, uint64_t seed, tm_ray *rays_out,
                           int64_t *count_dev, int32_t *src_out, void *stream) {
    if (!m || n < 0 || per_hit < 1 || per_hit > 1024 || !count_dev || (n > 0 && (!hits || !rays_out)))
        return TM_ERR_ARG;
    if ((((uintptr_t)rays_out) | ((uintptr_t)hits)) & 31u) return TM_ERR_ARG;
    if (!m->on_device) return TM_ERR_NO_DEVICE;
    if (n * (int64_t)per_hit > INT32_MAX) return TM_ERR_TOO_LARGE;
    return launch_gen_secondary(mesh_view(m), hits, n, n_dev, per_hit, tmax, seed, rays_out, count_dev,
                                src_out, (cudaStream_t)stream);
}

tm_status tm_gen_shadow(const tm_mesh *m, const tm_hit *hits, int64_t n, const int64_t *n_dev,
                        float lx, float ly, float lz, tm_ray *rays_out, int64_t *count_dev,
                        int32_t *src_out, void *stream) {
    if (!m || n < 0 || !count_dev || (n > 0 && (!hits || !rays_out))) return TM_ERR_ARG;
    if ((((uintptr_t)rays_out) | ((uintptr_t)hits)) & 31u) return TM_ERR_ARG;
    if (!(std::isfinite(lx) && std::isfinite(ly) && std::isfinite(lz))) return TM_ERR_ARG;
    if (!m->on_device) return TM_ERR_NO_DEVICE;
    if (n > INT32_MAX) return TM_ERR_TOO_LARGE;
    return launch_gen_shadow(mesh_view(m), hits, n, n_dev, lx, ly, lz, rays_out, count_dev, src_out,
                             (cudaStream_t)stream);
}

tm_status tm_gen_specular(const tm_mesh *m, const tm_ray *rays_in, const tm_hit *hits, int64_t n,
                          const int64_t *n_dev, int kind, float ior, float tmax, tm_ray *rays_out,
                          int64_t *count_dev, int32_t *src_out, void *stream) {
    if (!m || n < 0 || !count_dev || (n > 0 && (!hits || !rays_out || !rays_in))) return TM_ERR_ARG;
    if ((((uintptr_t)rays_out) | ((uintptr_t)hits) | ((uintptr_t)rays_in)) & 31u) return TM_ERR_ARG;
    if (kind != TM_SPECULAR_REFLECT && kind != TM_SPECULAR_REFRACT) return TM_ERR_ARG;
    if (!(ior > 0.f) || !std::isfinite(ior)) return TM_ERR_ARG;
    if (!m->on_device) return TM_ERR_NO_DEVICE;
    if (n > INT32_MAX) return TM_ERR_TOO_LARGE;
    return launch_gen_specular(mesh_view(m), rays_in, hits, n, n_dev, kind, ior, tmax, rays_out,
                               count_dev, src_out, (cudaStream_t)stream);
}

tm_status tm_gen_secondary_noalloc(const tm_mesh *m, const tm_hit *hits, int64_t n,
                                   const int64_t *n_dev, int per_hit, float tmax, uint64_t seed,
                                   tm_ray *rays_out, int64_t *count_dev, int32_t *src_out,
                                   void *stream) {
    if (!m || n < 0 || per_hit < 1 || per_hit > 1024 || !count_dev || (n > 0 && (!hits || !rays_out)))
        return TM_ERR_ARG;
    if ((((uintptr_t)rays_out) | ((uintptr_t)hits)) & 31u) return TM_ERR_ARG;
    if (!m->on_device) return TM_ERR_NO_DEVICE;
    if (n * (int64_t)per_hit > INT32_MAX) return TM_ERR_TOO_LARGE;
    return launch_gen_secondary_noalloc(mesh_view(m), hits, n, n_dev, per_hit, tmax, seed, rays_out,
                                        count_dev, src_out, (cudaStream_t)stream);
}

}  // extern "C"
