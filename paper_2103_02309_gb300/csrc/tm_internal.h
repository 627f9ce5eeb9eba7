// Internal declarations shared by the host build, the C ABI and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tetmesh.h"

// A neighbour field holds a tet id (bit 31 clear) or a flagged constrained
// face (Sec. 3: the top bit tells the two apart and the low 31 bits index a
// tet or a constrained face).  The mesh boundary is the flagged reserved id
// 0x7FFFFFFF.
#define TM_CFACE_FLAG 0x80000000u
#define TM_BOUNDARY 0xFFFFFFFFu

struct tm_mesh {
    int64_t np = 0, nt = 0, nc = 0;
    double extent = 0.0;
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    int32_t source_tet = 0;
    // host copies of the packed records
    std::vector<int32_t> tet16;  // nt*4: VX, NX0, NX1, NX2
    std::vector<int32_t> cold;   // nt*8: V0..V3 (positive orientation), N0..N3 (N_j across V_j)
    std::vector<float> pts4;     // np*4
    std::vector<int32_t> cface;  // nc*8: tri, tet+, tet-, 0, v0, v1, v2, 0
    std::vector<int32_t> cgeo;   // nc*12: {v0 xyz, tet+}, {v1 xyz, tri}, {v2 xyz, 0} (coordinates as float bits)
    std::vector<int32_t> restart; // nc*2*24: per triangle side, the tet there: V, N, vertex xyz, {T, skip}
    std::vector<int32_t> t20;    // nt*4: VX, N0, N1, N2 (neighbours by rank), when built
    std::vector<int32_t> t20n3;  // nt: N3, when built
    std::vector<int32_t> t20aos; // nt*5: VX, N0..N3 at a 20-byte stride, when built
    std::vector<int32_t> face;   // nt*32: four face entries {N, W, x, y, z, 0, 0, 0}, when built
    std::vector<int32_t> face16; // nt*16: four face entries {N | w << 29, x, y, z}, when built
    std::vector<int32_t> pperm, tperm;  // internal -> input
    std::vector<int32_t> pinv, tinv;    // input -> internal
    // device copies
    int device = -1;
    bool on_device = false;
    int4 *d_tet16 = nullptr;
    float4 *d_pts = nullptr;
    int4 *d_cold = nullptr;
    int4 *d_cface = nullptr;
    int4 *d_cgeo = nullptr;
    int4 *d_restart = nullptr;
    int32_t *d_seeds = nullptr;  // located tets of a kSeedGrid^3 lattice over the bounding box
    int4 *d_t20 = nullptr;
    int32_t *d_t20n3 = nullptr;
    int32_t *d_t20aos = nullptr;
    int4 *d_face = nullptr;
    int4 *d_face16 = nullptr;
    int64_t device_bytes = 0;
    int64_t n_regions = 0;  // regions found by TM_ORDER_HILBERT_REGIONS (else 0)
};

// Point location starts from the located tet of the nearest lattice point
// (a coarse grid of precomputed source tets) instead of one fixed source.
// 64^3 seeds (1 MB, located once when the mesh is uploaded): the camera's
// locate of a step took 7-8 us on GB300 against 12-14 us with 32^3.
constexpr int kSeedGrid = 64;

// What a kernel needs to walk one mesh.
struct MeshView {
    const int4 *tet16;
    const float4 *pts;
    const int4 *cold;
    const int4 *cface;
    const int4 *cgeo;      // three int4 per triangle: its vertices' coordinates and tet+ (hit geometry)
    const int4 *restart;   // six int4 per triangle side: the restart tet, inline (restarted rays)
    int32_t nt, np, nc;
    float extent;
    const int32_t *seeds;  // kSeedGrid^3 source tets for point location (may be null)
    const int4 *t20;       // Tet20 {VX, N0, N1, N2} (may be null)
    const int32_t *t20n3;  // Tet20 N3 (may be null)
    const int32_t *t20aos; // Tet20 packed {VX, N0..N3} (may be null)
    const int4 *face;      // face entries, two int4 each, four per tet (may be null)
    const int4 *face16;    // 16-byte face entries, four per tet (may be null)
    float lo[3], cell_inv;  // lattice origin and kSeedGrid / extent
    float hi[3];            // the points' bounding box is [lo, hi]
};

inline MeshView mesh_view(const tm_mesh *m) {
    MeshView v;
    v.tet16 = m->d_tet16;
    v.pts = m->d_pts;
    v.cold = m->d_cold;
    v.cface = m->d_cface;
    v.cgeo = m->d_cgeo;
    v.restart = m->d_restart;
    v.nt = (int32_t)m->nt;
    v.np = (int32_t)m->np;
    v.nc = (int32_t)m->nc;
    v.extent = (float)m->extent;
    v.seeds = m->d_seeds;
    v.t20 = m->d_t20;
    v.t20n3 = m->d_t20n3;
    v.t20aos = m->d_t20aos;
    v.face = m->d_face;
    v.face16 = m->d_face16;
    for (int a = 0; a < 3; ++a) {
        v.lo[a] = m->lo[a];
        v.hi[a] = m->hi[a];
    }
    v.cell_inv = m->extent > 0 ? (float)(kSeedGrid / m->extent) : 0.f;
    return v;
}

// Error text of the last CUDA failure (thread-local).
void tm_set_error(const char *what, cudaError_t e);
void tm_set_error_text(const std::string &s);
void tm_count_launches(uint64_t n);

#define TM_CUDA(call)                                   \
    do {                                                \
        cudaError_t _e = (call);                        \
        if (_e != cudaSuccess) {                        \
            tm_set_error(#call, _e);                    \
            return TM_ERR_CUDA;                         \
        }                                               \
    } while (0)

// Kernel launchers (defined in the .cu files).
struct TraceConfig {
    int mode;
    float tau;
    uint32_t max_steps;
    int block;
    int refill;
    int batch_steps;
    int ctas_per_sm;
    bool bounded;
    bool block_auto;  // block not given: two blocks an SM at the walk's register budget
    cudaEvent_t events[4];
    int format;
    const int32_t *stop_tet;  // point-light rays: DEVICE id of the tet to stop in (null: none); needs bounded
};
TraceConfig resolve_trace_opts(const tm_trace_opts *opts, int64_t nt);
// The record TM_FORMAT_AUTO walks: face entries when the mesh has them, else Tet32.
int auto_format(bool has_faces16, bool has_faces);

tm_status launch_trace(const MeshView &mv, const tm_ray *rays, int64_t n, const int64_t *n_dev,
                       tm_hit *hits, const TraceConfig &cfg, cudaStream_t s);
tm_status launch_locate(const MeshView &mv, const float *q, int64_t n, const int32_t *hint,
                        int32_t source, int32_t *out, uint32_t max_steps, cudaStream_t s);
tm_status launch_gen_primary(const tm_camera *cam, const int32_t *start, float tmax, tm_ray *rays,
                             cudaStream_t s);
tm_status launch_gen_secondary(const MeshView &mv, const tm_hit *hits, int64_t n,
                               const int64_t *n_dev, int per_hit, float tmax, uint64_t seed,
                               tm_ray *out, int64_t *count, int32_t *src, cudaStream_t s);

tm_status launch_gen_shadow(const MeshView &mv, const tm_hit *hits, int64_t n, const int64_t *n_dev,
                            float lx, float ly, float lz, tm_ray *out, int64_t *count, int32_t *src,
                            cudaStream_t s);
tm_status launch_gen_specular(const MeshView &mv, const tm_ray *rays_in, const tm_hit *hits,
                              int64_t n, const int64_t *n_dev, int kind, float ior, float tmax,
                              tm_ray *out, int64_t *count, int32_t *src, cudaStream_t s);

tm_status launch_gen_secondary_noalloc(const MeshView &mv, const tm_hit *hits, int64_t n,
                                       const int64_t *n_dev, int per_hit, float tmax, uint64_t seed,
                                       tm_ray *out, int64_t *count, int32_t *src, cudaStream_t s);

// Multi-mesh persistent trace over a device descriptor table.
struct BatchDesc {
    MeshView mesh;
    const tm_ray *rays;
    tm_hit *hits;
    const int32_t *perm;  // optional ray order (sorted), or null
    int64_t n;
    int64_t offset;       // first global ray index of this mesh
};
// `count`: add the launches to tm_launch_count (false while capturing a graph).
// `cursor` points to scratch of batch_scratch_bytes(total): the walk's ray
// counter (zeroed by the launcher).
inline size_t batch_scratch_bytes(int64_t) { return sizeof(unsigned long long); }
tm_status launch_trace_batch(const BatchDesc *descs_dev, int n_meshes, int64_t total,
                             const TraceConfig &cfg, unsigned long long *cursor, cudaStream_t s,
                             bool count);
int max_persistent_ctas(int mode, bool multi, bool bounded, int block, int *sm_count);
