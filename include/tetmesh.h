/*
 * tetmesh.h -- C ABI of the GB300 (sm_103a) library for ray traversal of a
 * constrained tetrahedral mesh, after Aman, Demirci & Gudukbay, "Compact
 * Tetrahedralization-based Acceleration Structure for Ray Tracing"
 * (arXiv 2103.02309).
 *
 * The library builds the compact mesh records of Sec. 3 (16-byte Tet16
 * records, the layout of the Tet16 figure, plus 16-byte aligned float4 points),
 * orders points and tets along a Hilbert curve (Sec. 5), locates points
 * with the walk of Sec. 4.2, and traces rays with the 2-D exit-face walk of
 * Sec. 4 (Alg. 1, Alg. 6-7, the scaled basis of Eq. 1-3 and the projected
 * origin of Sec. 7, optimisation 1), stopping at the first constrained face
 * it crosses (Sec. 3, last paragraph; Sec. 4).  Secondary
 * rays restart from a hit face into an adjacent tet (Sec. 6).
 *
 * Plain C types only: every pointer is either a host pointer or a CUDA
 * device pointer, as each function states; streams are cudaStream_t passed
 * as void*.  Device work is asynchronous on the given stream; the status a
 * function returns reports argument and launch errors only.  Per-ray
 * problems are reported in tm_hit.flags.  Functions are thread-safe for
 * distinct meshes; calls on one mesh from several host threads must be
 * serialised by the caller.
 *
 * Ids: tets and points are renumbered by tm_build (Hilbert order).  Tet ids
 * that the library returns (tm_hit.tet, tm_locate output) and that it takes
 * (tm_ray.start >= 0) are INTERNAL ids of that mesh; tm_map_ids converts
 * them to and from the caller's input ids.  Triangle ids are always the row
 * of the triangle in the caller's input; each input triangle is one
 * constrained face, so a constrained-face id equals its triangle id.
 */
#ifndef TETMESH_H
#define TETMESH_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tm_mesh tm_mesh;
typedef struct tm_batch tm_batch;

typedef enum {
    TM_OK = 0,
    TM_ERR_ARG = 1,              /* null pointer, negative count, bad option value */
    TM_ERR_RANGE = 2,            /* a vertex id outside [0, n_points) */
    TM_ERR_ORIENT = 3,           /* a tet with orient3d <= 0 (see tm_build) */
    TM_ERR_NONMANIFOLD = 4,      /* a face shared by more than two tets */
    TM_ERR_CFACE_UNMATCHED = 5,  /* a triangle that is not a face of any tet */
    TM_ERR_CFACE_DUPLICATE = 6,  /* two triangles on the same tet face */
    TM_ERR_OOM = 7,              /* host or device allocation failed */
    TM_ERR_CUDA = 8,             /* a CUDA call failed; see tm_last_error() */
    TM_ERR_TOO_LARGE = 9,        /* a count past an index range: more than 2^31-1 tets, points
                                    or rays, 2^30 triangles, 2^29 tets with 16-byte face
                                    entries, or the scratch-free generator's 2^24 hits */
    TM_ERR_NO_DEVICE = 10        /* the mesh was built without upload */
} tm_status;

/* Arithmetic of the traversal (Sec. 4; the guard is this library's). */
enum {
    TM_MODE_FP32_GUARD = 0, /* FP32 walk; a sign test whose |det| < tau*max|coord| is re-decided in FP64 */
    TM_MODE_FP32 = 1,       /* FP32 walk, no re-test */
    TM_MODE_FP64 = 2        /* FP64 projections and sign tests throughout */
};

/* Memory order of points and tets (Sec. 5): TM_ORDER_HILBERT sorts points
 * by the Hilbert key of their position and tets by that of their centroid;
 * TM_ORDER_INPUT keeps the input order; TM_ORDER_HILBERT_REGIONS sorts the
 * points the same way and the tets first by region, then by Hilbert key.  A
 * region is a maximal set of tets connected through faces that are not
 * constrained (a walk never leaves its region); regions are ordered by the
 * smallest Hilbert key of their tets. */
enum { TM_ORDER_HILBERT = 0, TM_ORDER_INPUT = 1, TM_ORDER_HILBERT_REGIONS = 2 };

/* Tet record the walk reads (Sec. 3): Tet16 = VX and NX_j = N_j ^ N_3
 * (16 B, decoded with the previous tet, Alg. 7); Tet20 = VX and N_0..N_3
 * sorted by the ids of the vertices they sit across (20 B, Alg. 5; needs
 * tm_build_opts.tet20), stored split (TM_FORMAT_TET20: a 16-B
 * {VX, N0, N1, N2} array and a 4-B N3 array) or packed (TM_FORMAT_TET20_AOS:
 * one int32[5] per tet at a 20-B stride); Tet32 = the full record V0..V3,
 * N0..N3 (32 B, the mesh's cold records, so it needs no extra memory; Alg. 3
 * with VX = V0^V1^V2^V3).  All give identical hits.  TM_FORMAT_AUTO (0)
 * selects the 16-byte face entries below when the mesh has them, else the
 * 32-byte ones, else Tet32: on
 * GB300 the walk is bound by instruction issue and cache latency, not by
 * HBM bandwidth, a 32-byte record costs one 32-byte sector like a 16-byte
 * one, and the full record needs the fewest instructions to decode.
 * TM_FORMAT_FACE (needs tm_build_opts.faces) is a layout of this library,
 * not one of the paper's records: per tet four 32-byte face entries, entry
 * r for the face opposite the vertex of rank r (vertex ids ascending), each
 * {N, W, x, y, z, 0, 0, 0}: the neighbour N across the face (flagged value
 * for a constrained face or the boundary) and the id W and float32 position
 * of N's vertex opposite that face (W = -1 when N is flagged).  A step then
 * needs one 32-byte read, issued as soon as the exit face is known, instead
 * of a record read followed by a dependent point read; it costs 128 B per
 * tet.  TM_FORMAT_FACE16 (needs tm_build_opts.faces16, at most 2^29 tets)
 * halves them: entry r is {N | w << 29, x, y, z} (16 B), with w the rank of
 * W among N's vertex ids in bits 29-30 of a tet value; the walk then tracks
 * the ranks of its face vertices instead of their ids.  Batches take Tet16,
 * Tet32, packed Tet20 or either face layout. */
enum {
    TM_FORMAT_AUTO = 0,
    TM_FORMAT_TET16 = 1,
    TM_FORMAT_TET20 = 2,
    TM_FORMAT_TET32 = 3,
    TM_FORMAT_TET20_AOS = 4,
    TM_FORMAT_FACE = 5,
    TM_FORMAT_FACE16 = 6
};

/* Ray and hit buffers (every tm_ray and tm_hit array passed to this
 * library) must be 32-byte aligned, as each record is 32 bytes and is read
 * and written whole; calls refuse other pointers with TM_ERR_ARG before any
 * launch. */

/* A ray, 32 bytes, two 16-byte words.
 *   start >= 0 : internal id of a tet that holds the origin (o).
 *   start <  0 : restart from a constrained face (Sec. 6): with
 *                code = -1 - start, the ray leaves triangle c = code >> 1 into
 *                the tet on side s = code & 1 of it (0: the side its normal
 *                (v1-v0) x (v2-v0) points to, in the triangle's input vertex
 *                order; 1: the other side) and cannot hit c itself.
 *   tmax       : hits with t > tmax are misses; +inf for unbounded rays.
 * t is measured in units of |d| (x(t) = o + t d); d need not be unit length. */
typedef struct {
    float ox, oy, oz;
    int32_t start;
    float dx, dy, dz;
    float tmax;
} tm_ray;

/* A hit, 32 bytes.  tri = -1 for a miss.  (b1, b2): barycentrics with
 * x = (1-b1-b2) v0 + b1 v1 + b2 v2 in the triangle's input vertex order.
 * tet: internal id of the tet the walk ended in (for a hit, the tet on the
 * arrival side of the triangle).  steps: tets entered after the start tet. */
typedef struct {
    int32_t tri;
    float t, b1, b2;
    int32_t tet;
    int32_t cface;
    uint32_t steps;
    uint32_t flags;
} tm_hit;

#define TM_HIT_SIDE_NEG   0x01u  /* the ray arrived from the - side of the hit triangle */
#define TM_HIT_STEP_LIMIT 0x02u  /* max_steps reached; reported as a miss */
#define TM_HIT_GUARD      0x04u  /* at least one sign test was re-decided in FP64 */
#define TM_HIT_BAD_START  0x08u  /* origin not in the start tet, an invalid restart face, or a
                                     ray without a line (d zero or not finite, o not finite);
                                     such a ray is a miss with tet -1 and steps 0 */
#define TM_HIT_TIE        0x10u  /* an exactly zero sign test was broken by vertex ids */
#define TM_HIT_FINAL_FP64 0x20u  /* t and barycentrics recomputed in FP64 */
#define TM_HIT_RESTART_3D 0x40u  /* a restart used the 3-D face-plane fallback step */
#define TM_HIT_BAD_ID     0x80u  /* an id read from the mesh was out of range (corrupt mesh); miss */
#define TM_HIT_START_MOVED 0x100u /* the origin lay on the start tet's boundary; the walk started
                                     in a neighbouring tet that also holds it */
#define TM_HIT_SLOW_PASS  0x200u  /* guard mode: at least one step had a sign test within the
                                     guard threshold and was re-decided out of line */
#define TM_HIT_REACHED    0x400u  /* tm_trace_shadow: the walk reached the light's tet (no
                                     constrained triangle in between); reported as a miss */

typedef struct {
    int32_t order;           /* TM_ORDER_* (default TM_ORDER_HILBERT) */
    int32_t fix_orientation; /* nonzero: swap V2,V3 of tets with orient3d < 0 instead of failing */
    int32_t tet20;           /* nonzero: also pack the Tet20 records, split and packed (40 B per tet) */
    int32_t faces;           /* nonzero: also pack the face entries of TM_FORMAT_FACE (128 B per tet) */
    int32_t faces16;         /* nonzero: also pack those of TM_FORMAT_FACE16 (64 B per tet) */
} tm_build_opts;

typedef struct {
    int32_t mode;        /* TM_MODE_* */
    float guard_tau;     /* relative guard threshold; <= 0 selects 1e-6 */
    uint32_t max_steps;  /* walk bound per ray; 0 selects 4*n_tets^(1/3)*8 + 256 */
    int32_t block;       /* threads per block: 0 (auto: two blocks an SM at the walk's register
                            budget), 64..1024, multiple of 32 */
    int32_t refill;      /* refill a warp once this many lanes are idle: 0 (auto), 1..32 */
    int32_t batch_steps; /* walk steps between refill checks: 0 (auto), 1..256 */
    int32_t ctas_per_sm; /* persistent CTAs per SM: 0 (as many as fit) */
    int32_t tmax_early_exit; /* nonzero: stop a walk once its entry face lies beyond t_max
                                (worth it for short rays, e.g. ambient occlusion) */
    void *phase_events[4];   /* optional cudaEvent_t handles recorded on the stream before the
                                start phase, after it, after the walk and after the finish
                                phase (tm_trace only); NULL entries are skipped */
    int32_t format;          /* TM_FORMAT_*: the record the walk reads (0: auto) */
} tm_trace_opts;

/* Mesh description returned by tm_mesh_info.  Device pointers are owned by
 * the mesh and valid until tm_destroy. */
typedef struct {
    int64_t n_points, n_tets, n_tris;
    double extent;               /* largest side of the points' bounding box */
    float bbox_lo[3], bbox_hi[3];
    int32_t source_tet;          /* default source tet of tm_locate (internal id) */
    int32_t on_device;           /* 1 after upload */
    const void *tet16_dev;       /* int4[n_tets]  (VX, NX0, NX1, NX2) */
    const void *points_dev;      /* float4[n_points] (x, y, z, 0) */
    const void *cold_dev;        /* int4[2*n_tets] (V0..V3 positively oriented, N0..N3) */
    const void *cface_dev;       /* int4[2*n_tris] (tri, tet+, tet-, 0, v0, v1, v2, 0) */
    const void *tet20_dev;       /* int4[n_tets] (VX, N0, N1, N2), or NULL */
    const void *tet20_n3_dev;    /* int32[n_tets] N3, or NULL */
    const void *tet20_aos_dev;   /* int32[5*n_tets] (VX, N0, N1, N2, N3), or NULL */
    const void *face_dev;        /* int32[32*n_tets] face entries (TM_FORMAT_FACE), or NULL */
    const void *face16_dev;      /* int32[16*n_tets] face entries (TM_FORMAT_FACE16), or NULL */
    int64_t device_bytes;        /* bytes the mesh holds on the device */
    int64_t n_regions;           /* regions found by TM_ORDER_HILBERT_REGIONS, else 0 */
} tm_mesh_info;

/* Builds the compact mesh (Sec. 3) from HOST arrays, which are copied:
 *   points  float32 [n_points*3] xyz,
 *   tets    int32 [n_tets*4] vertex ids, positively oriented
 *           (orient3d(V0,V1,V2,V3) = det[V1-V0, V2-V0, V3-V0] > 0),
 *   tris    int32 [n_tris*3] vertex ids of the constrained triangles; every
 *           triangle must be a face of one or two tets.
 * Steps: face matching (neighbours), constrained-face matching, Hilbert
 * reordering of points and tet centroids (Sec. 5), Tet16 packing with
 * neighbours sorted by their opposite vertex id (Sec. 3, Tet20/Tet16), the
 * cold full records used to start rays, and the constrained-face table
 * (Sec. 3: a flagged neighbour field indexes it; it keeps the triangle and
 * both adjacent tets).  upload != 0 also copies the records to the current
 * CUDA device.  On success *out owns everything; release with tm_destroy.
 * Errors: TM_ERR_ARG, TM_ERR_RANGE, TM_ERR_ORIENT, TM_ERR_NONMANIFOLD,
 * TM_ERR_CFACE_UNMATCHED, TM_ERR_CFACE_DUPLICATE, TM_ERR_TOO_LARGE,
 * TM_ERR_OOM, TM_ERR_CUDA; *out is NULL then. */
tm_status tm_build(const float *points, int64_t n_points, const int32_t *tets, int64_t n_tets,
                   const int32_t *tris, int64_t n_tris, const tm_build_opts *opts, int upload,
                   tm_mesh **out);

/* Releases a mesh and its device arrays (synchronises the device first). */
void tm_destroy(tm_mesh *mesh);

tm_status tm_mesh_info_get(const tm_mesh *mesh, tm_mesh_info *info);

/* Copies the packed host records into caller HOST buffers (any may be NULL):
 * tet16 int32[n_tets*4], cold int32[n_tets*8], points float32[n_points*4],
 * cface int32[n_tris*8], point_perm/tet_perm int32[n] (internal -> input id). */
tm_status tm_mesh_export(const tm_mesh *mesh, int32_t *tet16, int32_t *cold, float *points,
                         int32_t *cface, int32_t *point_perm, int32_t *tet_perm);

/* Copies the Tet20 records (when built) into HOST buffers: vxn
 * int32[n_tets*4] (VX, N0, N1, N2), n3 int32[n_tets] and aos int32[n_tets*5]
 * (VX, N0..N3); NULL buffers are skipped.  TM_ERR_ARG if the mesh was built
 * without them. */
tm_status tm_mesh_export_tet20(const tm_mesh *mesh, int32_t *vxn, int32_t *n3, int32_t *aos);

/* Copies the face entries (when built) into a HOST buffer int32[n_tets*32]
 * (the position words as float32 bit patterns).  TM_ERR_ARG if the mesh was
 * built without them. */
tm_status tm_mesh_export_faces(const tm_mesh *mesh, int32_t *faces);

/* The same for the 16-byte entries: faces16 int32[n_tets*16]. */
tm_status tm_mesh_export_faces16(const tm_mesh *mesh, int32_t *faces16);

/* Copies the restart records into a HOST buffer int32[n_tris*2*24]: for side
 * s of triangle c (record 2c + s, the index a restart ray's start field
 * names, Sec. 6) the tet on that side, {V0..V3}, {N0..N3} (its cold record),
 * the positions of V0..V3 (12 float32 bit patterns), then {T, skip, 0, 0}
 * with skip the local index of the face it shares with c; T = skip = -1 on a
 * side with no tet.  Always built. */
tm_status tm_mesh_export_restart(const tm_mesh *mesh, int32_t *restart);

enum { TM_IDS_TET = 0, TM_IDS_POINT = 1 };
enum { TM_TO_INPUT = 0, TM_TO_INTERNAL = 1 };
/* Converts n ids (HOST arrays) between internal and input numbering.  Ids
 * outside the valid range map to -1. */
tm_status tm_map_ids(const tm_mesh *mesh, int kind, int direction, const int32_t *in,
                     int32_t *out, int64_t n);

/* Point location (Sec. 4.2): for each DEVICE point q[i] (float32 xyz,
 * [n*3]) walks from a source tet's centroid along the segment to q[i] with
 * the 2-D exit-face test, crossing constrained faces, until the tet whose
 * exit plane lies beyond q[i]; writes its internal id to tet_out[i] (DEVICE
 * int32 [n]), or -1 when q[i] is outside the mesh or the walk exceeds its
 * bound.  hint (DEVICE int32 [n], may be NULL) gives a per-point source tet;
 * otherwise `source` (an internal id), or with source = -1 the located tet of
 * the nearest point of a 32^3 lattice over the bounding box (located once
 * when the mesh is uploaded), so that walks stay short. */
tm_status tm_locate(const tm_mesh *mesh, const float *q, int64_t n, const int32_t *hint,
                    int32_t source, int32_t *tet_out, void *stream);

/* Traces n DEVICE rays into n DEVICE hits (Sec. 4 + Sec. 7) in three
 * launches: per-ray start (basis, start-tet exit face or face restart), a
 * persistent walk whose warps refill idle lanes from a global ray cursor,
 * and per-ray finish (the hit); the hit buffer carries the per-ray state
 * between them.  If n_dev is not
 * NULL it points to a DEVICE int64 holding the ray count (read by the
 * kernel, clamped to n), so that counts produced on the device need no host
 * round trip.  opts may be NULL (defaults).  rays and hits must be 32-byte
 * aligned.  Errors: TM_ERR_ARG, TM_ERR_NO_DEVICE, TM_ERR_CUDA, and
 * TM_ERR_TOO_LARGE for n > 2^31 - 1 (refused before any buffer is read). */
tm_status tm_trace(const tm_mesh *mesh, const tm_ray *rays, int64_t n, const int64_t *n_dev,
                   tm_hit *hits, const tm_trace_opts *opts, void *stream);

/* Shadow rays toward a point light (Sec. 6): the walk of tm_trace, which
 * also ends, as a miss flagged TM_HIT_REACHED, when it enters (or starts in)
 * the tet that holds the light: *light_tet_dev (DEVICE int32, internal id,
 * e.g. written by tm_locate for the light at the start of the frame, so no
 * host round trip is needed).  A hit (tri >= 0) is the nearest constrained
 * triangle between the origin and the light: the light is occluded.  Each
 * ray's tmax should be its distance to the light (in units of |d|): a walk
 * that passes the light's tet by rounding then still ends, as a miss
 * without the flag, once its entry face lies beyond tmax
 * (opts->tmax_early_exit is implied).  A light tet id outside the mesh
 * (e.g. -1 from tm_locate for a light outside it) disables the stop.
 * Other arguments as tm_trace. */
tm_status tm_trace_shadow(const tm_mesh *mesh, const tm_ray *rays, int64_t n,
                          const int64_t *n_dev, const int32_t *light_tet_dev, tm_hit *hits,
                          const tm_trace_opts *opts, void *stream);

/* Pinhole camera of the synthetic workloads: eye, looking along +z, image x
 * along +x and image y (down) along -y; per pixel, with correctly rounded
 * float32 operations in this order (no fused multiply-add):
 *   sx = ((px+0.5)*kx - 1)*tx,  sy = (1 - (py+0.5)*ky)*ty,
 *   L = sqrt((sx*sx + sy*sy) + 1),  d = (sx/L, sy/L, 1/L),
 * rays stored in 8x4 pixel tiles, tiles row-major, pixels row-major inside
 * a tile (ragged edge tiles keep only in-image pixels). */
typedef struct {
    float eye[3];
    int32_t width, height;
    float kx, ky, tx, ty;  /* kx = 2/W, ky = 2/H, tx,ty = tan(fov/2) * side/shorter side */
} tm_camera;

/* Writes width*height primary rays (DEVICE tm_ray) starting in the tet
 * *start_dev (DEVICE int32, e.g. tm_locate's output for the eye). */
tm_status tm_gen_primary(const tm_camera *cam, const int32_t *start_dev, float tmax,
                         tm_ray *rays, void *stream);

/* Secondary rays from hits (Sec. 6): for every hit i (tri >= 0) of the n
 * DEVICE hits, `per_hit` rays leave the hit triangle back into the arrival
 * side's tet, with cosine-weighted directions about the triangle normal and
 * the given tmax.  Random numbers: SplitMix64 as a counter-based generator,
 * draw 2*(i*per_hit + k) + j of stream `seed`.  Output is compacted into
 * DEVICE rays_out (capacity n*per_hit) in 8 groups by the length of the
 * longest walk the hit's first ray can make (to the mesh's bounding box, or
 * to tmax), longest first, so that a walk over them takes its long rays
 * early and ends with a shorter tail.  Within a group, hits go by block of
 * 1024 consecutive hits, then by the octant of their first ray's direction
 * (bit 0: dx < 0, bit 1: dy < 0, bit 2: dz < 0), then in hit order, and the
 * per_hit rays of one hit are consecutive.  The order does not depend on
 * scheduling.  The count is written to DEVICE *count_dev
 * (int64), and src_out (DEVICE int32, may be NULL) gets the index i of each
 * ray's hit.  hits may hold n_dev (DEVICE int64, may be
 * NULL) valid entries instead of n.  A hit whose cface is not a constrained
 * face of this mesh (0 <= cface < n_tris fails: a foreign or corrupted
 * record) counts as a miss here and in the other generators. */
tm_status tm_gen_secondary(const tm_mesh *mesh, const tm_hit *hits, int64_t n,
                           const int64_t *n_dev, int per_hit, float tmax, uint64_t seed,
                           tm_ray *rays_out, int64_t *count_dev, int32_t *src_out, void *stream);

/* Shadow rays from hits (Sec. 6): for every hit i (tri >= 0) of the n
 * DEVICE hits, one ray from the hit point x = a + b1 (b - a) + b2 (c - a)
 * (triangle (a, b, c) in input order, float32) toward the point light
 * (lx, ly, lz): d = (L - x) / |L - x|, tmax = |L - x|, restarted from the
 * hit triangle into its side that faces the light (the + side when
 * ((b - a) x (c - a)) . (L - a) >= 0).  Output compacted in hit order
 * (capacity n); count, src_out and n_dev as tm_gen_secondary.  Trace them
 * with tm_trace_shadow. */
tm_status tm_gen_shadow(const tm_mesh *mesh, const tm_hit *hits, int64_t n, const int64_t *n_dev,
                        float lx, float ly, float lz, tm_ray *rays_out, int64_t *count_dev,
                        int32_t *src_out, void *stream);

/* Reflection and refraction rays from hits (Sec. 6): for every hit i
 * (tri >= 0) of the n DEVICE hits, made by ray i of rays_in, one ray from
 * the hit point (as tm_gen_shadow) with unit direction
 *   TM_SPECULAR_REFLECT: the mirror direction r = w + 2 c n_a, restarted
 *     into the arrival side's tet;
 *   TM_SPECULAR_REFRACT: the transmitted direction of Snell's law,
 *     t = eta w + (eta c - sqrt(k)) n_a with k = 1 - eta^2 (1 - c^2),
 *     restarted into the tet across the hit face; where k < 0 (total
 *     internal reflection) the mirror direction instead,
 * with w = d / |d| of the incoming ray, n_a the unit triangle normal turned
 * toward the arrival side, c = -w . n_a (clamped at 0), and eta the ratio of
 * refractive indices (arrival side over far side): ior for rays arriving
 * from the - side, 1/ior from the + side (ior = index of the - side over
 * that of the + side).  Output compacted in hit order (capacity n); count,
 * src_out and n_dev as tm_gen_secondary; all rays with the given tmax. */
enum { TM_SPECULAR_REFLECT = 0, TM_SPECULAR_REFRACT = 1 };
tm_status tm_gen_specular(const tm_mesh *mesh, const tm_ray *rays_in, const tm_hit *hits,
                          int64_t n, const int64_t *n_dev, int kind, float ior, float tmax,
                          tm_ray *rays_out, int64_t *count_dev, int32_t *src_out, void *stream);

/* The same as tm_gen_secondary, for callers that cannot allocate device
 * memory while they run (a renderer with a fixed memory budget, or code
 * inside a stream capture that must not add allocation nodes).  The paper
 * has no counterpart: this is a property of the library, not of the method.
 * It calls no cudaMalloc, cudaFree or allocating library routine: its scan
 * scratch is a static device array of this library, sized for at most
 * TM_NOALLOC_MAX_HITS hits (about 1.5 MiB, held on every device that loads
 * the library until the process exits).  n > TM_NOALLOC_MAX_HITS returns
 * TM_ERR_TOO_LARGE (tm_last_error() says why) and launches nothing.
 * The first call on each device looks up the array's device address and
 * keeps it for the life of the process; make that first call outside any
 * stream capture.  cudaDeviceReset (or any other teardown of the device's
 * primary context) unloads the library's module from that device and
 * leaves the kept address stale: do not call this function on a device
 * after resetting it in the same process.  All calls share the array,
 * so calls whose work overlaps on the GPU (several streams or host
 * threads) race on it: serialise them.  Nothing in the array needs to start
 * at zero; each call writes every entry it later reads. */
#define TM_NOALLOC_MAX_HITS (1 << 24)
tm_status tm_gen_secondary_noalloc(const tm_mesh *mesh, const tm_hit *hits, int64_t n,
                                   const int64_t *n_dev, int per_hit, float tmax, uint64_t seed,
                                   tm_ray *rays_out, int64_t *count_dev, int32_t *src_out,
                                   void *stream);

/* Batched, uneven multi-mesh tracing in one persistent launch (a work
 * queue over all rays of all meshes), replayed from a CUDA graph.
 * tm_batch_create: meshes (HOST array of n_meshes uploaded meshes).
 * tm_batch_set: HOST arrays of DEVICE ray/hit pointers and HOST counts; the
 *   descriptor table is uploaded synchronously and the graph is rebuilt.
 * tm_batch_run: replays the graph on `stream` (sort + trace).
 * tm_batch_run_separate: the same work as one tm_trace launch per mesh.
 * tm_batch_autotune: times candidate (format, block, refill, batch_steps,
 *   sort_chunk) settings on the current rays, keeps the fastest, and writes
 *   it to *best (may be NULL); sort_chunk 0 disables the ray sort. */
tm_status tm_batch_create(const tm_mesh *const *meshes, int n_meshes, tm_batch **out);
tm_status tm_batch_set(tm_batch *b, const tm_ray *const *rays, const int64_t *n,
                       tm_hit *const *hits, const tm_trace_opts *opts, int32_t sort_chunk);
tm_status tm_batch_run(tm_batch *b, void *stream);
tm_status tm_batch_run_separate(tm_batch *b, void *stream);
typedef struct {
    tm_trace_opts opts;
    int32_t sort_chunk;
    float ms;
} tm_tuned;
tm_status tm_batch_autotune(tm_batch *b, int reps, tm_tuned *best, void *stream);
void tm_batch_destroy(tm_batch *b);

/* Host utility: 3-D Hilbert index (Sec. 5's space-filling curve) of n
 * integer coordinates ijk (HOST uint32 [n*3], each < 2^bits, bits 1..21)
 * into keys (HOST uint64 [n]).  tm_build orders points and tet centroids by
 * these keys on a 2^21 grid over the bounding cube. */
tm_status tm_hilbert_keys(const uint32_t *ijk, int64_t n, int bits, uint64_t *keys);

/* Text of a status; text of the last CUDA error seen by this thread. */
const char *tm_status_str(tm_status s);
const char *tm_last_error(void);

/* Number of kernel launches this library has issued in this process (the
 * benchmark's launch count).  Graph replays count the kernels they hold. */
uint64_t tm_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* TETMESH_H */
