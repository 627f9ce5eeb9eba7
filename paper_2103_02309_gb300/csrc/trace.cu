// Ray traversal (Sec. 4 and Sec. 7 of the paper) for sm_103a, in three phases.
//
//  1. start_kernel, one thread per ray: scaled basis and projected origin
//     (Eq. 1-3, Sec. 7 optimisation 1), then the exit face of the start tet
//     with at most four 2-D triangle tests (Sec. 4), or the restart through a
//     hit face into the tet on its arrival side (Sec. 6).  It leaves a walk
//     record in the ray's own hit slot.
//  2. walk_kernel, persistent: the per-tet step (Alg. 1 on the new vertex,
//     then the neighbour across the exit face) until a flagged (constrained
//     or boundary) neighbour; it leaves an end record in the hit slot.  The
//     step reads one of the paper's records (Sec. 3), each with the float4
//     point of the new vertex:
//       Tet16 (Alg. 6-7): idx3 = idx0 ^ idx1 ^ idx2 ^ VX;
//         ra = rank of idx3, rb = rank of idx_exit among the four vertex ids;
//         N3 = ra == 3 ? prev : prev ^ NX_ra ;  next = rb == 3 ? N3 : N3 ^ NX_rb
//       Tet20 (Alg. 4-5): next = N[rb];  Tet32 (Alg. 2-3): next = N across idx_exit
//     or this library's face entries, which hold the neighbour across each
//     face together with the neighbour's new vertex, so a step is one read
//     issued once the exit face is known (16-byte entries keep the vertices'
//     ranks among the tet's ids instead of the ids).
//     Lanes whose ray ended are refilled from a global cursor once `refill`
//     lanes are idle (ballot + popc, one atomicAdd per warp, ids handed out
//     by rank within the idle mask), so the rays of one grab are consecutive
//     and warps stay full (the persistent-threads scheme of Aila & Laine,
//     "Understanding the efficiency of ray traversal on GPUs", HPG 2009).
//     In guard mode the walk makes the two sign tests Alg. 1 reads in
//     float32 and re-decides one that falls within the guard threshold in
//     double precision: the face-entry walks in the loop through an
//     out-of-line call; the walks over the paper's records park the ray in
//     its hit slot and re-decide the step at the lane's next refill, with no
//     walk state live across that call.
//     Bounded walks (short rays) also prefetch into L2, at each refill, the
//     records of the rays a little further along the cursor.
//  3. finish_kernel, one thread per ray: the ray-triangle test on the hit
//     triangle in its own vertex order (vertices read inline with the
//     triangle), with the FP64 guard, into the hit.  In guard mode a block
//     queues its ill-conditioned hits and redoes them in double precision
//     packed into full warps.
//
// Keeping the once-per-ray work out of the walk kernel keeps the walk's
// register state small and its code free of calls except the rare FP64
// re-test.  The hit slot (32 bytes per ray) carries the state between the
// phases, so no scratch memory is needed beyond the cursor.
#include <cmath>

#include "walk.cuh"

namespace tmk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxBatch = 64;

// The hit slot between the phases, 8 words:
//   [0] phase: 1 ended, 2 parked at tet [1] for a re-decided step; a walk
//       record (walk from here) holds -1 - (the tet the ray comes from),
//       which is negative, so that a bounded walk that ends before its first
//       step can name the tet its segment ends in whatever record it reads
//   [1] tet (walk: tet to enter; ended: last tet)
//   [2] walk: prev (Tet16 and the paper's other records) or the fourth vertex
//       of tet [1] (face entries); ended: the flagged value that ended the walk
//   [3..5] entry face ids, counter-clockwise in the ray's basis  [6] steps  [7] flags
constexpr int kPhaseEnded = 1, kPhaseParked = 2;
__device__ __forceinline__ int walk_phase(int32_t from) { return -1 - from; }
__device__ __forceinline__ bool is_walk_phase(int w) { return w < 0; }
__device__ __forceinline__ int32_t walk_from(int w) { return -1 - w; }

// A 32-byte slot written by one 256-bit store (sm_100 and later; the C ABI
// requires 32-byte aligned ray and hit buffers) instead of two 128-bit
// ones, so that L2 never receives a sector in halves.  Measured on GB300 in
// the start and finish phases and the ray generators: +0.4 % a step on the
// precision workload, +1.4 % on the large one.  The walk keeps two 128-bit
// stores: there the wide store (an asm statement the compiler cannot move
// loads across) made both walks 1-2 % slower.
#ifndef TM_ST256
#define TM_ST256 1
#endif
__device__ __forceinline__ void store32(void *p, const int4 &a, const int4 &b, bool streaming) {
    const unsigned long long q0 = ((unsigned long long)(uint32_t)a.y << 32) | (uint32_t)a.x;
    const unsigned long long q1 = ((unsigned long long)(uint32_t)a.w << 32) | (uint32_t)a.z;
    const unsigned long long q2 = ((unsigned long long)(uint32_t)b.y << 32) | (uint32_t)b.x;
    const unsigned long long q3 = ((unsigned long long)(uint32_t)b.w << 32) | (uint32_t)b.z;
    if (streaming)
        asm volatile("st.global.cs.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(q0), "l"(q1), "l"(q2),
                     "l"(q3) : "memory");
    else
        asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(q0), "l"(q1), "l"(q2),
                     "l"(q3) : "memory");
}

template <bool WIDE = false>
__device__ __forceinline__ void put_record(tm_hit *hp, int phase, int32_t tet, uint32_t prev_or_code,
                                           int32_t i0, int32_t i1, int32_t i2, uint32_t steps,
                                           uint32_t flags) {
    if (TM_ST256 && WIDE) {
        store32(hp, make_int4(phase, tet, (int)prev_or_code, i0), make_int4(i1, i2, (int)steps, (int)flags),
                false);
    } else {
        reinterpret_cast<int4 *>(hp)[0] = make_int4(phase, tet, (int)prev_or_code, i0);
        reinterpret_cast<int4 *>(hp)[1] = make_int4(i1, i2, (int)steps, (int)flags);
    }
}

template <bool WIDE = false>
__device__ __forceinline__ void put_end(tm_hit *hp, int32_t tet, uint32_t code, uint32_t steps,
                                        uint32_t flags) {
    put_record<WIDE>(hp, kPhaseEnded, tet, code, -1, -1, -1, steps, flags);
}

// Which mesh and which ray a global ray index names (batched launches).
struct Slot {
    int32_t m, local;
};
__device__ __forceinline__ Slot find_slot(const BatchDesc *d, int n_meshes, unsigned long long r) {
    int lo = 0, hi = n_meshes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((unsigned long long)d[mid].offset <= r) lo = mid; else hi = mid - 1;
    }
    return Slot{lo, (int32_t)(r - (unsigned long long)d[lo].offset)};
}

struct PhaseParams {
    int64_t n_cap;
    const int64_t *n_dev;
    float tau_rel;             // sign-test guard threshold relative to the mesh extent
    const int32_t *stop_tet;   // point-light rays: DEVICE id of the light's tet, else null
    int slot_i3;               // walk record word 2 = the next tet's fourth vertex (face entries)
};

// The light's tet of a shadow launch, or -1 (none, or not a tet of the mesh).
__device__ __forceinline__ int32_t load_stop(const int32_t *p, int32_t nt) {
    if (!p) return -1;
    const int32_t t = __ldg(p);
    return (t >= 0 && t < nt) ? t : -1;
}

__device__ __forceinline__ int64_t ray_count(const PhaseParams &P) {
    return P.n_dev ? min(P.n_cap, *P.n_dev) : P.n_cap;
}

// Rare start fallback: the origin lies on the boundary of the start tet and
// the line (with ties broken by vertex ids) does not pass through it.  Among
// the tets around it, up to two rings of face neighbours, returns the first
// that also holds the origin and that the line leaves through exactly one
// face; -1 if none.
template <int MODE>
__device__ __noinline__ int32_t search_start(const MeshView mv, const tm_ray *rp, int32_t T0,
                                             float tau) {
    typedef typename RealOf<MODE>::T R;
    const float4 w0 = __ldg(reinterpret_cast<const float4 *>(rp));
    const float4 w1 = __ldg(reinterpret_cast<const float4 *>(rp) + 1);
    const Basis<R> B = make_basis<R>(R(w1.x), R(w1.y), R(w1.z), R(w0.x), R(w0.y), R(w0.z));
    SignCtx sc;
    sc.ray = rp;
    sc.pts = mv.pts;
    sc.tau = tau;
    sc.flags = 0;
    int32_t tried[21];
    int n_tried = 0;
    tried[n_tried++] = T0;
    int32_t ring[4];
    const int4 n0 = __ldg(mv.cold + 2 * T0 + 1);
    ring[0] = n0.x; ring[1] = n0.y; ring[2] = n0.z; ring[3] = n0.w;
    for (int level = 0; level < 2; ++level) {
        int32_t cand[16];
        int nc = 0;
        if (level == 0) {
            for (int k = 0; k < 4; ++k) cand[nc++] = ring[k];
        } else {
            for (int k = 0; k < 4; ++k) {
                if (ring[k] < 0 || ring[k] >= mv.nt) continue;
                const int4 nn = __ldg(mv.cold + 2 * ring[k] + 1);
                cand[nc++] = nn.x; cand[nc++] = nn.y; cand[nc++] = nn.z; cand[nc++] = nn.w;
            }
        }
        for (int i = 0; i < nc; ++i) {
            const int32_t c = cand[i];
            if (c < 0 || c >= mv.nt) continue;  // flagged (constrained / boundary) or invalid
            bool seen = false;
            for (int j = 0; j < n_tried; ++j) seen |= tried[j] == c;
            if (seen || n_tried >= 21) continue;
            tried[n_tried++] = c;
            if (!holds_origin(mv, rp, c)) continue;
            WalkState<R> S;
            uint32_t next;
            if (line_init<MODE>(mv, B, c, -1, sc, S, next)) return c;
        }
    }
    return -1;
}

// Phase 1 for one ray.
template <int MODE>
__device__ __forceinline__ void start_one(const MeshView &mv, const tm_ray *rp, tm_hit *hp,
                                          float tau_rel, int32_t stop_tet, bool slot_i3) {
    typedef typename RealOf<MODE>::T R;
    const float4 w0 = __ldcs(reinterpret_cast<const float4 *>(rp));
    const float4 w1 = __ldcs(reinterpret_cast<const float4 *>(rp) + 1);
    const Basis<R> B = make_basis<R>(R(w1.x), R(w1.y), R(w1.z), R(w0.x), R(w0.y), R(w0.z));
    SignCtx sc;
    sc.ray = rp;
    sc.pts = mv.pts;
    sc.tau = tau_rel * mv.extent;
    sc.flags = 0;
    WalkState<R> S;
    uint32_t steps = 0;
    const int32_t start = __float_as_int(w0.w);
    uint32_t next = TM_BOUNDARY;
    int32_t T = -1;
    bool ok = false;
    // a ray without a line (a zero or non-finite direction, or a non-finite
    // origin) has no walk: it ends here as a flagged miss
    const bool line = isfinite(w0.x) && isfinite(w0.y) && isfinite(w0.z) && isfinite(w1.x) &&
                      isfinite(w1.y) && isfinite(w1.z) && (w1.x != 0.f || w1.y != 0.f || w1.z != 0.f);
    if (!line) {
    } else if (start >= 0) {
        if (start < mv.nt) {
            T = start;
            ok = line_init<MODE>(mv, B, T, -1, sc, S, next);
            if (!ok) {
                const int32_t T2 = search_start<MODE>(mv, rp, T, sc.tau);
                if (T2 >= 0) {
                    T = T2;
                    ok = line_init<MODE>(mv, B, T, -1, sc, S, next);
                    sc.flags |= TM_HIT_START_MOVED;
                }
            }
        }
    } else {
        const int32_t code = -1 - start;
        const int32_t c = code >> 1;
        int skip = -1;
        // the tet on the restart side, its entry face and its vertices, from
        // the side's restart record
        if (c < mv.nc) ok = restart_init<MODE>(mv, B, (int64_t)code, T, skip, sc, S, next);
        if (T >= 0) {
            if (skip >= 0) {
                for (int it = 0; !ok && it < 16; ++it) {
                    // the line misses T by rounding: one 3-D step, then retry
                    sc.flags |= TM_HIT_RESTART_3D;
                    const int2 st = step3d(mv, rp, T, skip);
                    const uint32_t nb = (uint32_t)st.x;
                    if (nb & TM_CFACE_FLAG) { next = nb; S.prev = T; ok = true; break; }
                    if (nb >= (uint32_t)mv.nt || st.y < 0) break;
                    ++steps;
                    T = (int32_t)nb;
                    skip = st.y;
                    ok = line_init<MODE>(mv, B, T, skip, sc, S, next);
                }
            } else {
                T = -1;
            }
        }
    }
    if (!ok)
        put_end<true>(hp, T, TM_BOUNDARY, steps, sc.flags | TM_HIT_BAD_START);
    else if (T == stop_tet)  // the ray starts in the light's tet: nothing lies in between
        put_end<true>(hp, T, TM_BOUNDARY, steps, sc.flags | TM_HIT_REACHED);
    else if (next & TM_CFACE_FLAG)
        put_end<true>(hp, S.prev, next, steps, sc.flags);
    else if ((int32_t)next == stop_tet)
        put_end<true>(hp, (int32_t)next, TM_BOUNDARY, steps, sc.flags | TM_HIT_REACHED);
    else if (slot_i3) {
        // the face-entry walk starts from the next tet's fourth vertex
        const int4 cv = __ldg(mv.cold + 2 * (int64_t)next);
        const int32_t i3 = cv.x ^ cv.y ^ cv.z ^ cv.w ^ S.i0 ^ S.i1 ^ S.i2;
        put_record<true>(hp, walk_phase(T), (int32_t)next, (uint32_t)i3, S.i0, S.i1, S.i2, steps, sc.flags);
    } else
        put_record<true>(hp, walk_phase(T), (int32_t)next, (uint32_t)S.prev, S.i0, S.i1, S.i2, steps,
                   sc.flags);
}

// The start phase chases three or four dependent reads per ray (the ray,
// its restart face, the tet's record and points, the next tet's record) and
// is latency-bound, so it wants warps in flight, but it also holds much
// state.  Measured on GB300 (start of camera / bounce / occlusion rays):
// three blocks of 256 an SM at 80 registers (72 bytes of spill) 12-18 %
// faster than four at 64 (368 bytes of spill: a ray's spills went to L2,
// three sectors each way) and than two at 104 (no spill, 16 warps).  (The
// double-precision arm, whose state is twice as wide, keeps its
// registers.)  The finish phase keeps four blocks an SM at 64 registers,
// which it fits without spilling.
#ifndef TM_START_MIN_BLOCKS
#define TM_START_MIN_BLOCKS 3
#endif
#ifndef TM_FINISH_MIN_BLOCKS
#define TM_FINISH_MIN_BLOCKS 4
#endif

template <int MODE, bool MULTI>
__global__ void __launch_bounds__(256, MODE == FP64 ? 1 : TM_START_MIN_BLOCKS)
start_kernel(const __grid_constant__ MeshView mv0, const tm_ray *__restrict__ rays0,
             tm_hit *__restrict__ hits0, const BatchDesc *__restrict__ descs, int n_meshes,
             const __grid_constant__ PhaseParams P) {
    const int64_t n = ray_count(P);
    const int32_t stop = MULTI ? -1 : load_stop(P.stop_tet, mv0.nt);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        if (MULTI) {
            const Slot s = find_slot(descs, n_meshes, (unsigned long long)r);
            const BatchDesc &D = descs[s.m];
            start_one<MODE>(D.mesh, D.rays + s.local, D.hits + s.local, P.tau_rel, -1, P.slot_i3 != 0);
        } else {
            start_one<MODE>(mv0, rays0 + r, hits0 + r, P.tau_rel, stop, P.slot_i3 != 0);
        }
    }
}

// In guard mode the float32 ray-triangle test is redone in double precision
// when its condition estimate (see mt_hit) exceeds kFinalCond, i.e. when the
// float32 t could be off by more than about 2e-6 relative.
constexpr float kFinalCond = 32.f;

// Phase 3 for one ray: the hit (or miss) from the end record.  In guard
// mode with `defer`, a hit whose float32 test is ill-conditioned is left
// untouched and reported (returns true), for a second call with `direct64`
// that goes straight to double precision.
template <int MODE>
__device__ __forceinline__ bool finish_one(const MeshView &mv, const tm_ray *rp, tm_hit *hp,
                                           bool defer = false, bool direct64 = false) {
    const int4 e0 = __ldcs(reinterpret_cast<const int4 *>(hp));
    const int4 e1 = __ldcs(reinterpret_cast<const int4 *>(hp) + 1);
    const int32_t tet = e0.y;
    uint32_t code = (uint32_t)e0.z;
    const uint32_t steps = (uint32_t)e1.z;
    uint32_t flags = (uint32_t)e1.w;
    if (e0.x != kPhaseEnded) {  // the walk never ended this ray (cannot happen for a completed launch)
        code = TM_BOUNDARY;
        flags |= TM_HIT_BAD_ID;
    }
    int32_t tri = -1, cf = -1;
    float t = __int_as_float(0x7f800000), b1 = 0.f, b2 = 0.f;
    if (code != TM_BOUNDARY && (int32_t)(code & ~TM_CFACE_FLAG) >= mv.nc) {
        flags |= TM_HIT_BAD_ID;
        code = TM_BOUNDARY;
    }
    if (code != TM_BOUNDARY) {
        const float4 w0 = __ldg(reinterpret_cast<const float4 *>(rp));
        const float4 w1 = __ldg(reinterpret_cast<const float4 *>(rp) + 1);
        const int32_t c = (int32_t)(code & ~TM_CFACE_FLAG);
        // the triangle's vertices inline: {a, tet+}, {b, tri}, {d, 0}
        const int4 g0 = __ldg(mv.cgeo + 3 * c), g1 = __ldg(mv.cgeo + 3 * c + 1),
                   g2 = __ldg(mv.cgeo + 3 * c + 2);
        const float4 a = make_float4(__int_as_float(g0.x), __int_as_float(g0.y), __int_as_float(g0.z), 0.f);
        const float4 b = make_float4(__int_as_float(g1.x), __int_as_float(g1.y), __int_as_float(g1.z), 0.f);
        const float4 d = make_float4(__int_as_float(g2.x), __int_as_float(g2.y), __int_as_float(g2.z), 0.f);
        float th, u, v;
        if (MODE == FP64) {
            double td, ud, vd, cd;
            mt_hit<double>(w0, w1, a, b, d, td, ud, vd, cd);
            th = (float)td; u = (float)ud; v = (float)vd;
        } else {
            float cond = 0.f;
            if (!(MODE == FP32G && direct64)) mt_hit<float>(w0, w1, a, b, d, th, u, v, cond);
            if (MODE == FP32G && (direct64 || !(cond <= kFinalCond))) {
                if (defer) return true;
                double td, ud, vd, cd;
                mt_hit<double>(w0, w1, a, b, d, td, ud, vd, cd);
                th = (float)td; u = (float)ud; v = (float)vd;
                flags |= TM_HIT_FINAL_FP64;
            }
        }
        if (th <= w1.w) {
            tri = g1.w;
            cf = c;
            t = th;
            b1 = u;
            b2 = v;
            if (g0.w != tet) flags |= TM_HIT_SIDE_NEG;
        }
    }
#if TM_ST256
    store32(hp, make_int4(tri, __float_as_int(t), __float_as_int(b1), __float_as_int(b2)),
            make_int4(tet, cf, (int)steps, (int)flags), true);
#else
    __stcs(reinterpret_cast<int4 *>(hp), make_int4(tri, __float_as_int(t), __float_as_int(b1),
                                                   __float_as_int(b2)));
    __stcs(reinterpret_cast<int4 *>(hp) + 1, make_int4(tet, cf, (int)steps, (int)flags));
#endif
    return false;
}

template <int MODE, bool MULTI>
__device__ __forceinline__ bool finish_at(const MeshView &mv0, const tm_ray *rays0, tm_hit *hits0,
                                          const BatchDesc *descs, int n_meshes, int64_t r,
                                          bool defer, bool direct64) {
    if (MULTI) {
        const Slot s = find_slot(descs, n_meshes, (unsigned long long)r);
        const BatchDesc &D = descs[s.m];
        return finish_one<MODE>(D.mesh, D.rays + s.local, D.hits + s.local, defer, direct64);
    }
    return finish_one<MODE>(mv0, rays0 + r, hits0 + r, defer, direct64);
}

constexpr int kFinishBlock = 256;
// Start and finish grids: at most this many 256-thread blocks per SM
// (grid-stride beyond), each a whole number of waves (three start blocks
// and four finish blocks fit an SM at once).  Measured on the precision
// workload: the start phases 4-6 % shorter at 24 than at 32; the finish
// phases 5 % longer at 24 than at 32, where each block takes one chunk of
// 1024 rays; 16 was 0.5 % slower a step than 32, and 256 slows the start.
#ifndef TM_START_CTAS_PER_SM
#define TM_START_CTAS_PER_SM 24
#endif
#ifndef TM_FINISH_CTAS_PER_SM
#define TM_FINISH_CTAS_PER_SM 32
#endif
#ifndef TM_FINISH_RAYS_PER_THREAD
#define TM_FINISH_RAYS_PER_THREAD 4
#endif
constexpr int kFinishChunk = kFinishBlock * TM_FINISH_RAYS_PER_THREAD;
// At the start of a chunk each thread pulls into L2 the end records (1), or
// the end records and the rays (2), of its later rays, so that their reads
// do not each wait on DRAM in turn.  Measured on GB300 (2): the finish
// phases 8 % faster on the precision workload and on the large scene's
// occlusion rays, though most of those end without a hit and never read
// their ray; (1) gained half of that.
#ifndef TM_FINISH_PREFETCH
#define TM_FINISH_PREFETCH 2
#endif

// In guard mode about one hit in twenty needs the double-precision test,
// and on GB300's narrow FP64 pipe a warp pays for it if any of its lanes
// does.  So each block first finishes a chunk of rays in float32 (four a
// thread), queues the ill-conditioned ones in shared memory, then redoes
// those packed into full warps: about two warps of double-precision work
// per 1024 rays instead of some 25.
template <int MODE, bool MULTI>
__global__ void __launch_bounds__(kFinishBlock, MODE == FP64 ? 1 : TM_FINISH_MIN_BLOCKS)
finish_kernel(const __grid_constant__ MeshView mv0, const tm_ray *__restrict__ rays0,
              tm_hit *__restrict__ hits0, const BatchDesc *__restrict__ descs, int n_meshes,
              const __grid_constant__ PhaseParams P) {
    const int64_t n = ray_count(P);
    if constexpr (MODE == FP32G) {
        __shared__ int queue[kFinishChunk];
        __shared__ int queued;
        // block-uniform trip count: every thread reaches every barrier
        for (int64_t base = blockIdx.x * (int64_t)kFinishChunk; base < n;
             base += (int64_t)gridDim.x * kFinishChunk) {
            if (threadIdx.x == 0) queued = 0;
            if (TM_FINISH_PREFETCH && !MULTI) {
                for (int j = threadIdx.x + kFinishBlock; j < kFinishChunk; j += kFinishBlock) {
                    const int64_t r = base + j;
                    if (r < n) {
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(hits0 + r));
                        if (TM_FINISH_PREFETCH > 1) asm volatile("prefetch.global.L2 [%0];" ::"l"(rays0 + r));
                    }
                }
            }
            __syncthreads();
            for (int j = threadIdx.x; j < kFinishChunk; j += kFinishBlock) {
                const int64_t r = base + j;
                if (r < n && finish_at<MODE, MULTI>(mv0, rays0, hits0, descs, n_meshes, r, true, false))
                    queue[atomicAdd(&queued, 1)] = j;
            }
            __syncthreads();
            for (int q = threadIdx.x; q < queued; q += kFinishBlock)
                finish_at<MODE, MULTI>(mv0, rays0, hits0, descs, n_meshes, base + queue[q], false, true);
            __syncthreads();
        }
    } else {
        for (int64_t r = blockIdx.x * (int64_t)kFinishBlock + threadIdx.x; r < n;
             r += (int64_t)gridDim.x * kFinishBlock)
            finish_at<MODE, MULTI>(mv0, rays0, hits0, descs, n_meshes, r, false, false);
    }
}

template <class R, bool BOUNDED> struct Depth {
    __device__ __forceinline__ void init(const float4 &, const float4 &) {}
    __device__ __forceinline__ void set(int, const float4 &) {}
    __device__ __forceinline__ bool far(const float4 &) const { return false; }
    __device__ __forceinline__ void put(int, bool) {}
    __device__ __forceinline__ bool beyond() const { return false; }
};
template <class R> struct Depth<R, true> {
    // whether each entry-face vertex lies beyond t_max along the ray (bit k
    // for slot k): three bits instead of three depths keep the bounded walk's
    // state small
    R dx, dy, dz, dod, zmax;
    uint32_t bits;
    __device__ __forceinline__ void init(const float4 &w0, const float4 &w1) {
        dx = w1.x; dy = w1.y; dz = w1.z;
        dod = rfma(dz, R(w0.z), rfma(dy, R(w0.y), rmul(dx, R(w0.x))));
        zmax = R(w1.w) * rfma(dz, dz, rfma(dy, dy, rmul(dx, dx)));
        bits = 0;
    }
    __device__ __forceinline__ R depth(const float4 &p) const {
        return rfma(dz, R(p.z), rfma(dy, R(p.y), rmul(dx, R(p.x)))) - dod;
    }
    __device__ __forceinline__ bool far(const float4 &p) const { return depth(p) > zmax; }
    __device__ __forceinline__ void put(int slot, bool b) {
        bits = (bits & ~(1u << slot)) | ((uint32_t)b << slot);
    }
    __device__ __forceinline__ void set(int slot, const float4 &p) { put(slot, far(p)); }
    // the entry face of the next tet lies entirely beyond t_max
    __device__ __forceinline__ bool beyond() const { return bits == 7u; }
};

// One tet record in the walk's format, and the decode of the neighbour across
// the exit vertex ie (Sec. 3 and Alg. 3, 5, 7).  i0..i2 are the entry face,
// i3 the new vertex; prev is the tet the walk came from.
// `base` is the format's record array of the mesh (rec_base); the split
// Tet20 layout also reads its second array from the mesh view.
template <int FMT> struct TetRec;

template <int FMT> __device__ __forceinline__ const int4 *rec_base(const MeshView &mv) {
    return FMT == TM_FORMAT_FACE16 ? mv.face16
         : FMT == TM_FORMAT_FACE ? mv.face
         : FMT == TM_FORMAT_TET32 ? mv.cold
         : FMT == TM_FORMAT_TET20 ? mv.t20
         : FMT == TM_FORMAT_TET20_AOS ? reinterpret_cast<const int4 *>(mv.t20aos)
                                      : mv.tet16;
}

template <> struct TetRec<TM_FORMAT_TET16> {  // VX, NX_j = N_j ^ N_3, neighbours by vertex rank
    int4 r;
    __device__ __forceinline__ void load(const MeshView &, const int4 *base, int32_t t) {
        r = __ldg(base + t);
    }
    __device__ __forceinline__ int32_t vx() const { return r.x; }
    __device__ __forceinline__ uint32_t next(int32_t prev, int32_t i0, int32_t i1, int32_t i2,
                                             int32_t i3, int32_t ie) const {
        const int ra = (i0 < i3) + (i1 < i3) + (i2 < i3);
        const int rb = (i0 < ie) + (i1 < ie) + (i2 < ie) + (i3 < ie);
        const uint32_t nxa = ra == 0 ? r.y : (ra == 1 ? r.z : (ra == 2 ? r.w : 0));
        const uint32_t nxb = rb == 0 ? r.y : (rb == 1 ? r.z : (rb == 2 ? r.w : 0));
        return (uint32_t)prev ^ nxa ^ nxb;
    }
};

template <> struct TetRec<TM_FORMAT_TET20> {  // VX, N_0..N_3 by vertex rank
    int4 r;
    int32_t n3;
    __device__ __forceinline__ void load(const MeshView &mv, const int4 *base, int32_t t) {
        r = __ldg(base + t);
        n3 = __ldg(mv.t20n3 + t);
    }
    __device__ __forceinline__ int32_t vx() const { return r.x; }
    __device__ __forceinline__ uint32_t next(int32_t, int32_t i0, int32_t i1, int32_t i2, int32_t i3,
                                             int32_t ie) const {
        const int rb = (i0 < ie) + (i1 < ie) + (i2 < ie) + (i3 < ie);
        return (uint32_t)(rb == 0 ? r.y : (rb == 1 ? r.z : (rb == 2 ? r.w : n3)));
    }
};

template <> struct TetRec<TM_FORMAT_TET20_AOS> {  // the same, packed at a 20-byte stride
    int32_t vx_, n[4];
    __device__ __forceinline__ void load(const MeshView &, const int4 *base, int32_t t) {
        const int32_t *p = reinterpret_cast<const int32_t *>(base) + 5 * (int64_t)t;
        vx_ = __ldg(p);
        n[0] = __ldg(p + 1);
        n[1] = __ldg(p + 2);
        n[2] = __ldg(p + 3);
        n[3] = __ldg(p + 4);
    }
    __device__ __forceinline__ int32_t vx() const { return vx_; }
    __device__ __forceinline__ uint32_t next(int32_t, int32_t i0, int32_t i1, int32_t i2, int32_t i3,
                                             int32_t ie) const {
        const int rb = (i0 < ie) + (i1 < ie) + (i2 < ie) + (i3 < ie);
        return (uint32_t)(rb == 0 ? n[0] : (rb == 1 ? n[1] : (rb == 2 ? n[2] : n[3])));
    }
};

// One 32-byte record in a single 256-bit load (sm_100 and later; the cold
// records are 32-byte aligned), or as two 128-bit loads.
#ifndef TM_LD256
#define TM_LD256 1
#endif
__device__ __forceinline__ void load32(const int4 *p, int4 &a, int4 &b) {
#if TM_LD256
    // four 64-bit lanes (the eight-word form of the same load stops this
    // toolchain's compiler on this kernel)
    unsigned long long q0, q1, q2, q3;
    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];" : "=l"(q0), "=l"(q1), "=l"(q2), "=l"(q3) : "l"(p));
    a = make_int4((int)(uint32_t)q0, (int)(q0 >> 32), (int)(uint32_t)q1, (int)(q1 >> 32));
    b = make_int4((int)(uint32_t)q2, (int)(q2 >> 32), (int)(uint32_t)q3, (int)(q3 >> 32));
#else
    a = __ldg(p);
    b = __ldg(p + 1);
#endif
}

template <> struct TetRec<TM_FORMAT_TET32> {  // V_0..V_3 and N_j across V_j (the cold record)
    int4 v, nb;
    __device__ __forceinline__ void load(const MeshView &, const int4 *base, int32_t t) {
        load32(base + 2 * (int64_t)t, v, nb);
    }
    __device__ __forceinline__ int32_t vx() const { return v.x ^ v.y ^ v.z ^ v.w; }
    __device__ __forceinline__ uint32_t next(int32_t, int32_t, int32_t, int32_t, int32_t,
                                             int32_t ie) const {
        return (uint32_t)(ie == v.x ? nb.x : (ie == v.y ? nb.y : (ie == v.z ? nb.z : nb.w)));
    }
};

struct WalkParams {
    int64_t n_cap;
    const int64_t *n_dev;
    unsigned long long *cursor;  // the walk's ray counter
    uint32_t max_steps;
    float tau_rel;
    int refill;
    int batch_steps;
    const int32_t *stop_tet;  // point-light rays (bounded walks only): DEVICE light tet, else null
};

// Guard mode: one step of a parked ray, with the double-precision re-test of
// the sign tests that fell within the threshold (the float32 walk left it
// undecided).  Reads the walk record from the hit slot and writes back the
// record of the next tet, or the end record.  Out of line: no walk state is
// live across the call, so the walk loop keeps its small register budget.
template <int FMT, bool BOUNDED>
__device__ __noinline__ void resolve_parked(const MeshView mv, const tm_ray *rp, tm_hit *hp,
                                            float tau_rel, uint32_t max_steps, int32_t stop_tet) {
    typedef float R;
    const int4 a = __ldcg(reinterpret_cast<const int4 *>(hp));
    const int4 b = __ldcg(reinterpret_cast<const int4 *>(hp) + 1);
    WalkState<R> S;
    S.tet = a.y;
    S.prev = a.z;
    S.i0 = a.w;
    S.i1 = b.x;
    S.i2 = b.y;
    uint32_t steps = (uint32_t)b.z;
    SignCtx sc;
    sc.ray = rp;
    sc.pts = mv.pts;
    sc.tau = tau_rel * mv.extent;
    sc.flags = (uint32_t)b.w | TM_HIT_SLOW_PASS;
    const float4 w0 = __ldg(reinterpret_cast<const float4 *>(rp));
    const float4 w1 = __ldg(reinterpret_cast<const float4 *>(rp) + 1);
    const Basis<R> B = make_basis<R>(w1.x, w1.y, w1.z, w0.x, w0.y, w0.z);
    const float4 x0 = __ldg(mv.pts + S.i0), x1 = __ldg(mv.pts + S.i1), x2 = __ldg(mv.pts + S.i2);
    S.p0 = B.project(x0.x, x0.y, x0.z);
    S.p1 = B.project(x1.x, x1.y, x1.z);
    S.p2 = B.project(x2.x, x2.y, x2.z);
    S.m0 = guard_mag(S.p0, sc.tau);
    S.m1 = guard_mag(S.p1, sc.tau);
    S.m2 = guard_mag(S.p2, sc.tau);
    // the face-entry walk re-decides from the full record (same neighbours)
    constexpr int RF = (FMT == TM_FORMAT_FACE || FMT == TM_FORMAT_FACE16) ? TM_FORMAT_TET32 : FMT;
    TetRec<RF> rec;
    rec.load(mv, rec_base<RF>(mv), S.tet);
    const int32_t i3 = S.i0 ^ S.i1 ^ S.i2 ^ rec.vx();
    if ((uint32_t)i3 >= (uint32_t)mv.np) {
        put_end(hp, S.tet, TM_BOUNDARY, steps, sc.flags | TM_HIT_BAD_ID);
        return;
    }
    const float4 x = __ldg(mv.pts + i3);
    const P2<R> p3 = B.project(x.x, x.y, x.z);
    const float m3 = guard_mag(p3, sc.tau);
    const int e = exit_slot_bits(step_signs<FP32G, false, true>(S, p3, i3, m3, sc));
    const int32_t ie = e == 0 ? S.i0 : (e == 1 ? S.i1 : S.i2);
    const uint32_t next = rec.next(S.prev, S.i0, S.i1, S.i2, i3, ie);
    float4 xf[3] = {x0, x1, x2};
    if (e == 0) S.i0 = i3; else if (e == 1) S.i1 = i3; else S.i2 = i3;
    xf[e] = x;
    ++steps;
    if (next & TM_CFACE_FLAG) {
        put_end(hp, S.tet, next, steps, sc.flags);
    } else if (next >= (uint32_t)mv.nt) {
        put_end(hp, S.tet, TM_BOUNDARY, steps, sc.flags | TM_HIT_BAD_ID);
    } else if (steps >= max_steps) {
        put_end(hp, S.tet, TM_BOUNDARY, steps, sc.flags | TM_HIT_STEP_LIMIT);
    } else if (BOUNDED && next == (uint32_t)stop_tet) {
        put_end(hp, (int32_t)next, TM_BOUNDARY, steps, sc.flags | TM_HIT_REACHED);
    } else {
        if (BOUNDED) {
            Depth<R, true> Z;
            Z.init(w0, w1);
            Z.set(0, xf[0]);
            Z.set(1, xf[1]);
            Z.set(2, xf[2]);
            if (Z.beyond()) {
                put_end(hp, S.tet, TM_BOUNDARY, steps, sc.flags);
                return;
            }
        }
        uint32_t w2 = (uint32_t)S.tet;
        if (FMT == TM_FORMAT_FACE || FMT == TM_FORMAT_FACE16) {  // as the start phase writes it
            const int4 cv = __ldg(mv.cold + 2 * (int64_t)next);
            w2 = (uint32_t)(cv.x ^ cv.y ^ cv.z ^ cv.w ^ S.i0 ^ S.i1 ^ S.i2);
        }
        put_record(hp, walk_phase(S.tet), (int32_t)next, w2, S.i0, S.i1, S.i2, steps, sc.flags);
    }
}

// Register budget per thread of the walk (float32; the FP64 arm keeps
// double-width state).  An SM's 65,536 registers hold 36 warps at 56
// registers a thread against 32 at 64; measured on GB300, the extra warps
// hide more of the bounce rays' record latency (bounce walk -8 %) and cost
// the guard mode a few bytes of spill.  48 registers spill more and lose.
#ifndef TM_WALK_MAXREG
#define TM_WALK_MAXREG 56
#endif
// Guard mode: the face-entry walk re-decides an ambiguous step in the loop
// with the out-of-line double-precision triple product (1); the walks over
// the paper's records park the ray and re-decide the step at the lane's next
// refill.  Measured on GB300: in the loop the face-entry walk is 5 % faster,
// while the Tet32 walk, whose loop holds more state, spills and loses 15 %.
#ifndef TM_GUARD_IN_LOOP
#define TM_GUARD_IN_LOOP 1
#endif
// 16-byte face entries: the four vertex ranks packed as bytes of one
// register (1) or kept in four (0), per mode.  Measured on GB300: packing
// frees registers around the guard's call and makes the guarded walk 6 %
// faster, while the pure float32 walk is faster unpacked.
#ifndef TM_PACKED_RANKS_GUARD
#define TM_PACKED_RANKS_GUARD 1
#endif
#ifndef TM_PACKED_RANKS_OTHER
#define TM_PACKED_RANKS_OTHER 0
#endif
template <int MODE> struct PackedRanks {
    static constexpr bool value = MODE == FP32G ? TM_PACKED_RANKS_GUARD : TM_PACKED_RANKS_OTHER;
};
template <int FMT> struct GuardInLoop {
    static constexpr bool value = TM_GUARD_IN_LOOP && (FMT == TM_FORMAT_FACE || FMT == TM_FORMAT_FACE16);
};

// Guard mode, 16-byte face entries: the walk keeps the ranks of its
// vertices among the current tet's ids, so the re-test of one sign test
// (ranks ra = the new vertex, rb = a face vertex) first recovers the ids from
// the tet's full record.  Returns bit 0 = det(p_a, p_b) > 0 by the
// double-precision triple product (ties by ids, which order like the ranks),
// TM_HIT_GUARD / TM_HIT_TIE in bits 8 and up.  Out of line.
__device__ __noinline__ static uint32_t guard_pair_ranked(const tm_ray *ray, const float4 *pts,
                                                          const int4 *cold, int32_t tet, int ra,
                                                          int rb) {
    const int4 cv = __ldg(cold + 2 * (int64_t)tet);
    const int32_t V[4] = {cv.x, cv.y, cv.z, cv.w};
    int32_t id[4] = {0, 0, 0, 0};
    for (int j = 0; j < 4; ++j)
        id[(V[0] < V[j]) + (V[1] < V[j]) + (V[2] < V[j]) + (V[3] < V[j])] = V[j];
    const float4 w0 = __ldg(reinterpret_cast<const float4 *>(ray));
    const float4 w1 = __ldg(reinterpret_cast<const float4 *>(ray) + 1);
    const double dd = triple(w0, w1, __ldg(pts + id[ra]), __ldg(pts + id[rb]));
    if (dd != 0.0) return (uint32_t)(dd > 0.0) | (TM_HIT_GUARD << 8);
    return (uint32_t)(id[ra] < id[rb]) | ((TM_HIT_GUARD | TM_HIT_TIE) << 8);
}
#ifndef TM_WALK_MAXREG_FP64
#define TM_WALK_MAXREG_FP64 72
#endif
// Bounded walks (early exit at t_max) carry the ray's depth state as well.
// On short ambient-occlusion rays 64 registers (32 warps an SM) measured
// 13 % faster than 80 (24 warps) and 4 % faster than 72 or 56.
#ifndef TM_WALK_MAXREG_BOUNDED
#define TM_WALK_MAXREG_BOUNDED 64
#endif

// How far ahead of a refill's rays (in rays) bounded walks prefetch records.
constexpr unsigned long long kRefillPrefetchAhead = 1024;

constexpr int walk_maxreg(int mode, bool bounded) {
    return mode == FP64 ? TM_WALK_MAXREG_FP64 : (bounded ? TM_WALK_MAXREG_BOUNDED : TM_WALK_MAXREG);
}

// Default threads per block: two blocks an SM with as many warps as the
// register budget allows (65,536 registers an SM, 64 warps at most):
// 576 threads at 56 registers, 512 at 64.  The double-precision arm is
// bound by the FP64 pipe instead: 512 threads (one block, 16 warps an SM at
// 72 registers) measured 2 % faster than two blocks of 448.
int walk_default_block(int mode, bool bounded) {
    if (mode == FP64) return 512;
    int warps = 65536 / (walk_maxreg(mode, bounded) * 32);
    if (warps > 64) warps = 64;
    return warps / 2 * 32;
}

template <int MODE, int FMT, bool BOUNDED, bool MULTI>
__global__ void __maxnreg__(walk_maxreg(MODE, BOUNDED))
walk_kernel(const __grid_constant__ MeshView mv0, const tm_ray *__restrict__ rays0,
            tm_hit *__restrict__ hits0, const BatchDesc *__restrict__ descs, int n_meshes,
            const __grid_constant__ WalkParams P) {
    typedef typename RealOf<MODE>::T R;
    extern __shared__ BatchDesc sdesc[];
    if (MULTI) {
        for (int i = threadIdx.x; i < n_meshes; i += blockDim.x) sdesc[i] = descs[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    int64_t n = P.n_cap;
    if (P.n_dev) n = min(n, *P.n_dev);

    bool active = false, parked = false, pool_empty = false;
    int32_t m = 0;
    tm_hit *hp = nullptr;
    const int4 *recs = rec_base<FMT>(mv0);
    const float4 *pts = mv0.pts;
    WalkState<R> S;
    Basis<R> B;
    Depth<R, BOUNDED> Z;
    SignCtx sc;
    sc.ray = nullptr;
    sc.pts = pts;
    sc.tau = P.tau_rel * mv0.extent;
    sc.flags = 0;
    uint32_t steps = 0;
    const int32_t stop = (BOUNDED && !MULTI) ? load_stop(P.stop_tet, mv0.nt) : -1;
    bool far3 = false;  // face entries, bounded walks: the current tet's fourth vertex lies beyond t_max

    for (;;) {
        bool load = false;
        if (MODE == FP32G && parked) {
            // re-decide the step this lane parked, then go on from its new record
            resolve_parked<FMT, BOUNDED>(MULTI ? sdesc[m].mesh : mv0, sc.ray, hp, P.tau_rel,
                                         P.max_steps, stop);
            parked = false;
            load = true;
        }
        const unsigned idle = __ballot_sync(kFull, !active && !load);
        const int n_idle = __popc(idle);
        if (!pool_empty && n_idle >= P.refill) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(P.cursor, (unsigned long long)n_idle);
            base = __shfl_sync(kFull, base, 0);
            if (base + (unsigned long long)n_idle >= (unsigned long long)n) pool_empty = true;
            const unsigned long long r = base + __popc(idle & ((1u << lane) - 1u));
            if (!active && !load && r < (unsigned long long)n) {
                int32_t local;
                if (MULTI) {
                    const Slot s = find_slot(sdesc, n_meshes, r);
                    m = s.m;
                    local = sdesc[m].perm ? sdesc[m].perm[s.local] : s.local;
                    recs = rec_base<FMT>(sdesc[m].mesh);
                    pts = sdesc[m].mesh.pts;
                    sc.ray = sdesc[m].rays + local;
                    sc.pts = pts;
                    sc.tau = P.tau_rel * sdesc[m].mesh.extent;
                    hp = sdesc[m].hits + local;
                } else {
                    local = (int32_t)r;
                    sc.ray = rays0 + local;
                    hp = hits0 + local;
                }
                load = true;
            }
            if (BOUNDED && !MULTI) {
                // Short bounded rays (ambient occlusion, shadows) refill
                // often, and the start phase wrote their records long enough
                // ago for them to have left L2: pull the records of the rays
                // some warp will take a little later into L2 now.  Measured
                // on GB300: the AO walk 3 % faster; unbounded walks, which
                // refill rarely, lose a little to the extra instructions.
                const unsigned long long rq = base + kRefillPrefetchAhead + (unsigned long long)lane;
                if (lane < n_idle && rq < (unsigned long long)n) {
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(hits0 + rq));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(rays0 + rq));
                }
            }
        }
        if (load) {
            // the walk record and the ray in one round trip
            const int4 a = __ldcg(reinterpret_cast<const int4 *>(hp));
            const int4 b = __ldcg(reinterpret_cast<const int4 *>(hp) + 1);
            const float4 w0 = __ldg(reinterpret_cast<const float4 *>(sc.ray));
            const float4 w1 = __ldg(reinterpret_cast<const float4 *>(sc.ray) + 1);
            if (is_walk_phase(a.x)) {
                S.tet = a.y;
                S.prev = a.z;
                S.i0 = a.w;
                S.i1 = b.x;
                S.i2 = b.y;
                steps = (uint32_t)b.z;
                sc.flags = (uint32_t)b.w;
                B = make_basis<R>(R(w1.x), R(w1.y), R(w1.z), R(w0.x), R(w0.y), R(w0.z));
                const float4 x0 = __ldg(pts + S.i0), x1 = __ldg(pts + S.i1), x2 = __ldg(pts + S.i2);
                S.p0 = B.project(R(x0.x), R(x0.y), R(x0.z));
                S.p1 = B.project(R(x1.x), R(x1.y), R(x1.z));
                S.p2 = B.project(R(x2.x), R(x2.y), R(x2.z));
                if (MODE == FP32G) {
                    S.m0 = guard_mag(S.p0, sc.tau);
                    S.m1 = guard_mag(S.p1, sc.tau);
                    S.m2 = guard_mag(S.p2, sc.tau);
                }
                active = true;
                if (BOUNDED) {
                    Z.init(w0, w1);
                    Z.set(0, x0);
                    Z.set(1, x1);
                    Z.set(2, x2);
                    if (Z.beyond()) {  // the segment ends in the tet the ray comes from
                        put_end(hp, walk_from(a.x), TM_BOUNDARY, steps, sc.flags);
                        active = false;
                    }
                }
                if ((FMT == TM_FORMAT_FACE || FMT == TM_FORMAT_FACE16) && active) {
                    // the fourth vertex of the tet entered (written by the start phase)
                    S.i3 = a.z;
                    if ((uint32_t)S.i3 >= (uint32_t)(MULTI ? sdesc[m].mesh.np : mv0.np)) {
                        put_end(hp, S.tet, TM_BOUNDARY, steps, sc.flags | TM_HIT_BAD_ID);
                        active = false;
                    } else {
                        const float4 x3 = __ldg(pts + S.i3);
                        S.p3 = B.project(R(x3.x), R(x3.y), R(x3.z));
                        if (MODE == FP32G) S.m3 = guard_mag(S.p3, sc.tau);
                        if (BOUNDED) far3 = Z.far(x3);
                        if (FMT == TM_FORMAT_FACE16) {
                            // from here on the walk keeps ranks among the tet's ids
                            const int32_t j0 = S.i0, j1 = S.i1, j2 = S.i2, j3 = S.i3;
                            S.i0 = (j1 < j0) + (j2 < j0) + (j3 < j0);
                            S.i1 = (j0 < j1) + (j2 < j1) + (j3 < j1);
                            S.i2 = (j0 < j2) + (j1 < j2) + (j3 < j2);
                            S.i3 = (j0 < j3) + (j1 < j3) + (j2 < j3);
                            if (PackedRanks<MODE>::value)  // bytes 0..2: the face slots, byte 3: the fourth vertex
                                S.i0 = S.i0 | (S.i1 << 8) | (S.i2 << 16) | (S.i3 << 24);
                        }
                    }
                }
            }
        }
        if (!__any_sync(kFull, active || parked)) {
            if (pool_empty) break;
            continue;
        }
        for (int k = 0; k < P.batch_steps; ++k) {
            if (!active) continue;
            if constexpr (FMT == TM_FORMAT_FACE16) {
                // ---- one step over 16-byte face entries, on vertex ranks ----
                const uint32_t PR = (uint32_t)S.i0;  // packed ranks (PackedRanks)
                const int q0 = PackedRanks<MODE>::value ? (int)(PR & 0xffu) : S.i0;
                const int q1 = PackedRanks<MODE>::value ? (int)((PR >> 8) & 0xffu) : S.i1;
                const int q2 = PackedRanks<MODE>::value ? (int)((PR >> 16) & 0xffu) : S.i2;
                const int q3 = PackedRanks<MODE>::value ? (int)(PR >> 24) : S.i3;
                int e;
                if constexpr (MODE == FP32G) {
                // Alg. 1 reads two sign tests: det(p3, p0), then det(p3, p1) when it
                // is positive, det(p3, p2) otherwise; only those two are guarded
                const R d0 = det2_packed(S.p3, S.p0);
                bool s0 = d0 > R(0);
                if (MODE == FP32G) {
                    if (!(fabsf((float)d0) > fmaxf(S.m3, S.m0))) {
                        const uint32_t r = guard_pair_ranked(sc.ray, pts, MULTI ? sdesc[m].mesh.cold : mv0.cold,
                                                             S.tet, q3, q0);
                        sc.flags |= r >> 8;
                        s0 = r & 1u;
                    }
                }
                const P2<R> pk = s0 ? S.p1 : S.p2;
                const R dk = det2_packed(S.p3, pk);
                bool sk = dk > R(0);
                if (MODE == FP32G) {
                    if (!(fabsf((float)dk) > fmaxf(S.m3, s0 ? S.m1 : S.m2))) {
                        const uint32_t r = guard_pair_ranked(sc.ray, pts, MULTI ? sdesc[m].mesh.cold : mv0.cold,
                                                             S.tet, q3, s0 ? q1 : q2);
                        sc.flags |= r >> 8;
                        sk = r & 1u;
                    }
                }
                e = s0 ? (sk ? 0 : 2) : (sk ? 1 : 0);
                } else {
                // unguarded: the three sign tests, exact zeros broken by ranks
                // (they order like the ids they stand for)
                const R d0 = det2(S.p3, S.p0), d1 = det2(S.p3, S.p1), d2 = det2(S.p3, S.p2);
                uint32_t sig = (uint32_t)(d0 > R(0)) | ((uint32_t)(d1 > R(0)) << 1) |
                               ((uint32_t)(d2 > R(0)) << 2);
                if ((d0 == R(0)) | (d1 == R(0)) | (d2 == R(0))) {
                    sc.flags |= TM_HIT_TIE;
                    if (d0 == R(0)) sig |= (uint32_t)(q3 < q0);
                    if (d1 == R(0)) sig |= (uint32_t)(q3 < q1) << 1;
                    if (d2 == R(0)) sig |= (uint32_t)(q3 < q2) << 2;
                }
                e = exit_slot_bits(sig);
                }
                const int re = PackedRanks<MODE>::value ? (int)((PR >> (8 * e)) & 0xffu)
                                               : (e == 0 ? S.i0 : (e == 1 ? S.i1 : S.i2));
                const int4 f = __ldg(recs + 4 * (int64_t)S.tet + re);
                if (PackedRanks<MODE>::value) {
                    const int sh = 8 * e;
                    S.i0 = (int32_t)((PR & ~(0xffu << sh)) | ((PR >> 24) << sh));
                    if (e == 0) { S.p0 = S.p3; S.m0 = S.m3; }
                    else if (e == 1) { S.p1 = S.p3; S.m1 = S.m3; }
                    else { S.p2 = S.p3; S.m2 = S.m3; }
                } else {
                    if (e == 0) { S.i0 = S.i3; S.p0 = S.p3; S.m0 = S.m3; }
                    else if (e == 1) { S.i1 = S.i3; S.p1 = S.p3; S.m1 = S.m3; }
                    else { S.i2 = S.i3; S.p2 = S.p3; S.m2 = S.m3; }
                }
                if (BOUNDED) Z.put(e, far3);
                ++steps;
                const uint32_t enc = (uint32_t)f.x;
                const uint32_t next = (enc & TM_CFACE_FLAG) ? enc : (enc & 0x1FFFFFFFu);
                uint32_t code = next;
                bool done = false;
                if (next >= (uint32_t)(MULTI ? sdesc[m].mesh.nt : mv0.nt)) {
                    done = true;
                    if (!(next & TM_CFACE_FLAG)) {
                        code = TM_BOUNDARY;
                        sc.flags |= TM_HIT_BAD_ID;
                    }
                } else if (steps >= P.max_steps) {
                    done = true;
                    code = TM_BOUNDARY;
                    sc.flags |= TM_HIT_STEP_LIMIT;
                } else if (BOUNDED && next == (uint32_t)stop) {
                    done = true;
                    code = TM_BOUNDARY;
                    sc.flags |= TM_HIT_REACHED;
                    S.tet = (int32_t)next;
                } else if (BOUNDED && Z.beyond()) {
                    done = true;
                    code = TM_BOUNDARY;
                } else {
                    // ranks in the next tet: the exit vertex leaves, W enters at rank w
                    const int w = (int)((enc >> 29) & 3u);
                    if (PackedRanks<MODE>::value) {
                        // per byte (values 0..3, no carries): r - [r > re], then + [r' >= w]
                        uint32_t F = (uint32_t)S.i0 & 0x00ffffffu;
                        F -= ((F + (0x007f7f7fu - (uint32_t)re * 0x010101u)) >> 7) & 0x010101u;
                        F += ((F + (0x80u - (uint32_t)w) * 0x010101u) >> 7) & 0x010101u;
                        S.i0 = (int32_t)(F | ((uint32_t)w << 24));
                    } else {
                        int r = S.i0; r -= (r > re); S.i0 = r + (r >= w);
                        r = S.i1; r -= (r > re); S.i1 = r + (r >= w);
                        r = S.i2; r -= (r > re); S.i2 = r + (r >= w);
                        S.i3 = w;
                    }
                    S.tet = (int32_t)next;
                    const float4 x3 = make_float4(__int_as_float(f.y), __int_as_float(f.z),
                                                  __int_as_float(f.w), 0.f);
                    S.p3 = B.project(R(x3.x), R(x3.y), R(x3.z));
                    if (MODE == FP32G) S.m3 = guard_mag(S.p3, sc.tau);
                    if (BOUNDED) far3 = Z.far(x3);
                }
                if (done) {
                    put_end(hp, S.tet, code, steps, sc.flags);
                    active = false;
                }
            } else if constexpr (FMT == TM_FORMAT_FACE) {
                // ---- one step over face entries: Alg. 1 on the vertex known
                // since entering the tet, then one 32-byte read ----
                const uint32_t sig = step_signs<MODE, MODE == FP32G && !GuardInLoop<FMT>::value, false>(S, S.p3, S.i3, S.m3, sc);
                if (MODE == FP32G && !GuardInLoop<FMT>::value && sig == kParked) {
                    put_record(hp, kPhaseParked, S.tet, (uint32_t)S.i3, S.i0, S.i1, S.i2, steps, sc.flags);
                    active = false;
                    parked = true;
                    continue;
                }
                const int e = exit_slot_bits(sig);
                const int32_t ie = e == 0 ? S.i0 : (e == 1 ? S.i1 : S.i2);
                const int rb = (S.i0 < ie) + (S.i1 < ie) + (S.i2 < ie) + (S.i3 < ie);
                int4 fa, fb;
                load32(recs + 2 * (4 * (int64_t)S.tet + rb), fa, fb);
                if (e == 0) { S.i0 = S.i3; S.p0 = S.p3; S.m0 = S.m3; }
                else if (e == 1) { S.i1 = S.i3; S.p1 = S.p3; S.m1 = S.m3; }
                else { S.i2 = S.i3; S.p2 = S.p3; S.m2 = S.m3; }
                if (BOUNDED) Z.put(e, far3);
                ++steps;
                const uint32_t next = (uint32_t)fa.x;
                uint32_t code = next;
                bool done = false;
                if (next >= (uint32_t)(MULTI ? sdesc[m].mesh.nt : mv0.nt)) {
                    // flagged values (bit 31) end the walk; other ids past the end are corrupt
                    done = true;
                    if (!(next & TM_CFACE_FLAG)) {
                        code = TM_BOUNDARY;
                        sc.flags |= TM_HIT_BAD_ID;
                    }
                } else if (steps >= P.max_steps) {
                    done = true;
                    code = TM_BOUNDARY;
                    sc.flags |= TM_HIT_STEP_LIMIT;
                } else if (BOUNDED && next == (uint32_t)stop) {
                    done = true;
                    code = TM_BOUNDARY;
                    sc.flags |= TM_HIT_REACHED;
                    S.tet = (int32_t)next;
                } else if (BOUNDED && Z.beyond()) {
                    done = true;
                    code = TM_BOUNDARY;
                } else {
                    S.tet = (int32_t)next;  // (the face-entry walk needs no previous tet)
                    S.i3 = fa.y;
                    const float4 x3 = make_float4(__int_as_float(fa.z), __int_as_float(fa.w),
                                                  __int_as_float(fb.x), 0.f);
                    S.p3 = B.project(R(x3.x), R(x3.y), R(x3.z));
                    if (MODE == FP32G) S.m3 = guard_mag(S.p3, sc.tau);
                    if (BOUNDED) far3 = Z.far(x3);
                }
                if (done) {
                    put_end(hp, S.tet, code, steps, sc.flags);
                    active = false;
                }
            } else {
            // ---- one step of Alg. 6 / Alg. 7 (or Alg. 4-5, Alg. 2-3) ----
            TetRec<FMT> rec;
            rec.load(mv0, recs, S.tet);
            const int32_t i3 = S.i0 ^ S.i1 ^ S.i2 ^ rec.vx();
            uint32_t code = TM_BOUNDARY;
            bool done = false;
            if ((uint32_t)i3 >= (uint32_t)(MULTI ? sdesc[m].mesh.np : mv0.np)) {
                // a corrupt record: end the ray instead of reading out of bounds
                done = true;
                sc.flags |= TM_HIT_BAD_ID;
            } else {
                const float4 x = __ldg(pts + i3);
                const P2<R> p3 = B.project(R(x.x), R(x.y), R(x.z));
                const float m3 = MODE == FP32G ? guard_mag(p3, sc.tau) : 0.f;
                const uint32_t sig = step_signs<MODE, MODE == FP32G, false>(S, p3, i3, m3, sc);
                if (MODE == FP32G && sig == kParked) {
                    // undecided in float32: park the ray; the lane re-decides this
                    // step out of line at its next refill
                    put_record(hp, kPhaseParked, S.tet, (uint32_t)S.prev, S.i0, S.i1, S.i2, steps, sc.flags);
                    active = false;
                    parked = true;
                    continue;
                }
                const int e = exit_slot_bits(sig);
                const int32_t ie = e == 0 ? S.i0 : (e == 1 ? S.i1 : S.i2);
                const uint32_t next = rec.next(S.prev, S.i0, S.i1, S.i2, i3, ie);
                if (e == 0) { S.i0 = i3; S.p0 = p3; S.m0 = m3; }
                else if (e == 1) { S.i1 = i3; S.p1 = p3; S.m1 = m3; }
                else { S.i2 = i3; S.p2 = p3; S.m2 = m3; }
                if (BOUNDED) Z.set(e, x);
                ++steps;
                code = next;
                if (next & TM_CFACE_FLAG) {
                    done = true;
                } else if (next >= (uint32_t)(MULTI ? sdesc[m].mesh.nt : mv0.nt)) {
                    done = true;
                    code = TM_BOUNDARY;
                    sc.flags |= TM_HIT_BAD_ID;
                } else if (steps >= P.max_steps) {
                    done = true;
                    code = TM_BOUNDARY;
                    sc.flags |= TM_HIT_STEP_LIMIT;
                } else if (BOUNDED && next == (uint32_t)stop) {
                    // reached the tet that holds the point light (Sec. 6)
                    done = true;
                    code = TM_BOUNDARY;
                    sc.flags |= TM_HIT_REACHED;
                    S.tet = (int32_t)next;
                } else if (BOUNDED && Z.beyond()) {
                    done = true;
                    code = TM_BOUNDARY;
                } else {
                    S.prev = S.tet;
                    S.tet = (int32_t)next;
                }
            }
            if (done) {
                put_end(hp, S.tet, code, steps, sc.flags);
                active = false;
            }
            }  // record formats
        }
    }
}

}  // namespace tmk

using namespace tmk;

namespace {

int sm_count_cached() {
    static int count = 0;
    if (count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&count, cudaDevAttrMultiProcessorCount, dev);
        if (count <= 0) count = 1;
    }
    return count;
}

template <int MODE, int FMT, bool BOUNDED, bool MULTI>
int walk_occupancy(int block, size_t smem) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, walk_kernel<MODE, FMT, BOUNDED, MULTI>, block,
                                                  smem);
    return nb;
}

template <bool BOUNDED, bool MULTI>
int occupancy_mode(int mode, int block, size_t smem) {
    switch (mode) {
        case FP32G: return walk_occupancy<FP32G, TM_FORMAT_TET16, BOUNDED, MULTI>(block, smem);
        case FP32: return walk_occupancy<FP32, TM_FORMAT_TET16, BOUNDED, MULTI>(block, smem);
        default: return walk_occupancy<FP64, TM_FORMAT_TET16, BOUNDED, MULTI>(block, smem);
    }
}

// Launches start, walk and finish for one mode.
template <int MODE, int FMT, bool BOUNDED, bool MULTI>
cudaError_t launch_phases(const MeshView &mv, const tm_ray *rays, tm_hit *hits, const BatchDesc *descs,
                          int n_meshes, const WalkParams &W, int block, int walk_grid,
                          const cudaEvent_t *ev, cudaStream_t s) {
    PhaseParams P;
    P.n_cap = W.n_cap;
    P.n_dev = W.n_dev;
    P.tau_rel = W.tau_rel;
    P.stop_tet = MULTI ? nullptr : W.stop_tet;
    P.slot_i3 = FMT == TM_FORMAT_FACE || FMT == TM_FORMAT_FACE16;
    const int sms = sm_count_cached();
    const int64_t g1 = (W.n_cap + 255) / 256;
    const int64_t g = std::min<int64_t>(g1, (int64_t)sms * TM_START_CTAS_PER_SM);
    const int64_t gmax = (int64_t)sms * TM_FINISH_CTAS_PER_SM;
    if (ev && ev[0]) cudaEventRecord(ev[0], s);
    start_kernel<MODE, MULTI><<<(int)g, 256, 0, s>>>(mv, rays, hits, descs, n_meshes, P);
    if (ev && ev[1]) cudaEventRecord(ev[1], s);
    const size_t smem = MULTI ? sizeof(BatchDesc) * (size_t)n_meshes : 0;
    walk_kernel<MODE, FMT, BOUNDED, MULTI><<<walk_grid, block, smem, s>>>(mv, rays, hits, descs,
                                                                           n_meshes, W);
    if (ev && ev[2]) cudaEventRecord(ev[2], s);
    int64_t gf = std::min<int64_t>(g1, gmax);
    if (MODE == FP32G) gf = std::min<int64_t>((W.n_cap + kFinishChunk - 1) / kFinishChunk, gmax);
    finish_kernel<MODE, MULTI><<<(int)gf, kFinishBlock, 0, s>>>(mv, rays, hits, descs, n_meshes, P);
    if (ev && ev[3]) cudaEventRecord(ev[3], s);
    return cudaGetLastError();
}

template <int FMT, bool BOUNDED, bool MULTI>
cudaError_t dispatch_fmt(int mode, const MeshView &mv, const tm_ray *rays, tm_hit *hits,
                         const BatchDesc *descs, int n_meshes, const WalkParams &W, int block,
                         int grid, const cudaEvent_t *ev, cudaStream_t s) {
    switch (mode) {
        case FP32G: return launch_phases<FP32G, FMT, BOUNDED, MULTI>(mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
        case FP32: return launch_phases<FP32, FMT, BOUNDED, MULTI>(mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
        default: return launch_phases<FP64, FMT, BOUNDED, MULTI>(mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
    }
}

template <bool BOUNDED, bool MULTI>
cudaError_t dispatch(int mode, int format, const MeshView &mv, const tm_ray *rays, tm_hit *hits,
                     const BatchDesc *descs, int n_meshes, const WalkParams &W, int block, int grid,
                     const cudaEvent_t *ev, cudaStream_t s) {
    if constexpr (MULTI) {  // batches: formats with one record array per mesh
        switch (format) {
            case TM_FORMAT_TET32: return dispatch_fmt<TM_FORMAT_TET32, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
            case TM_FORMAT_TET20_AOS: return dispatch_fmt<TM_FORMAT_TET20_AOS, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
            case TM_FORMAT_FACE: return dispatch_fmt<TM_FORMAT_FACE, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
            case TM_FORMAT_FACE16: return dispatch_fmt<TM_FORMAT_FACE16, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
            default: return dispatch_fmt<TM_FORMAT_TET16, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
        }
    } else {
        switch (format) {
            case TM_FORMAT_TET20: return dispatch_fmt<TM_FORMAT_TET20, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
            case TM_FORMAT_TET32: return dispatch_fmt<TM_FORMAT_TET32, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
            case TM_FORMAT_TET20_AOS: return dispatch_fmt<TM_FORMAT_TET20_AOS, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
            case TM_FORMAT_FACE: return dispatch_fmt<TM_FORMAT_FACE, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
            case TM_FORMAT_FACE16: return dispatch_fmt<TM_FORMAT_FACE16, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
            default: return dispatch_fmt<TM_FORMAT_TET16, BOUNDED, MULTI>(mode, mv, rays, hits, descs, n_meshes, W, block, grid, ev, s);
        }
    }
}

}  // namespace

int max_persistent_ctas(int mode, bool multi, bool bounded, int block, int *sm_count) {
    const int sms = sm_count_cached();
    if (sm_count) *sm_count = sms;
    const size_t smem = multi ? sizeof(BatchDesc) * kMaxBatch : 0;
    int per_sm;
    if (multi) per_sm = occupancy_mode<false, true>(mode, block, smem);
    else if (bounded) per_sm = occupancy_mode<true, false>(mode, block, smem);
    else per_sm = occupancy_mode<false, false>(mode, block, smem);
    return per_sm > 0 ? per_sm : 1;
}

TraceConfig resolve_trace_opts(const tm_trace_opts *o, int64_t nt) {
    TraceConfig c;
    c.mode = o ? o->mode : TM_MODE_FP32_GUARD;
    c.tau = (o && o->guard_tau > 0.f) ? o->guard_tau : 1e-6f;
    const double side = std::cbrt((double)(nt > 0 ? nt : 1));
    c.max_steps = (o && o->max_steps) ? o->max_steps : (uint32_t)(4.0 * side * 8.0 + 256.0);
    c.refill = (o && o->refill) ? o->refill : 4;
    c.batch_steps = (o && o->batch_steps) ? o->batch_steps : 16;
    c.ctas_per_sm = o ? o->ctas_per_sm : 0;
    c.bounded = o ? o->tmax_early_exit != 0 : false;
    c.block_auto = !(o && o->block);
    c.block = c.block_auto ? walk_default_block(c.mode, c.bounded) : o->block;
    for (int i = 0; i < 4; ++i) c.events[i] = o ? (cudaEvent_t)o->phase_events[i] : nullptr;
    c.format = o ? o->format : TM_FORMAT_AUTO;  // resolved against the mesh at launch
    c.stop_tet = nullptr;
    return c;
}

static bool valid_config(const TraceConfig &c) {
    return (c.mode == FP32G || c.mode == FP32 || c.mode == FP64) &&
           (c.format == TM_FORMAT_TET16 || c.format == TM_FORMAT_TET20 || c.format == TM_FORMAT_TET32 ||
            c.format == TM_FORMAT_TET20_AOS || c.format == TM_FORMAT_FACE ||
            c.format == TM_FORMAT_FACE16) &&
           c.block >= 32 &&
           c.block <= 1024 && c.block % 32 == 0 && c.refill >= 1 && c.refill <= 32 &&
           c.batch_steps >= 1 && c.batch_steps <= 256 && c.ctas_per_sm >= 0;
}

int auto_format(bool has_faces16, bool has_faces) {
    return has_faces16 ? TM_FORMAT_FACE16 : (has_faces ? TM_FORMAT_FACE : TM_FORMAT_TET32);
}

tm_status launch_trace(const MeshView &mv, const tm_ray *rays, int64_t n, const int64_t *n_dev,
                       tm_hit *hits, const TraceConfig &cfg_in, cudaStream_t s) {
    TraceConfig cfg = cfg_in;
    if (cfg.format == TM_FORMAT_AUTO) cfg.format = auto_format(mv.face16 != nullptr, mv.face != nullptr);
    if (cfg.block_auto) cfg.block = walk_default_block(cfg.mode, cfg.bounded);
    if (!valid_config(cfg)) return TM_ERR_ARG;
    if (n == 0) return TM_OK;
    if (n > INT32_MAX) return TM_ERR_TOO_LARGE;
    unsigned long long *cursor = nullptr;  // the walk's ray counter
    TM_CUDA(cudaMallocAsync((void **)&cursor, sizeof(unsigned long long), s));
    const cudaError_t ez = cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s);
    if (ez != cudaSuccess) {
        cudaFreeAsync(cursor, s);
        tm_set_error("cudaMemsetAsync (ray cursor)", ez);
        return TM_ERR_CUDA;
    }
    WalkParams W;
    W.n_cap = n;
    W.n_dev = n_dev;
    W.cursor = cursor;
    W.max_steps = cfg.max_steps;
    W.tau_rel = cfg.tau;
    W.refill = cfg.refill;
    W.batch_steps = cfg.batch_steps;
    W.stop_tet = cfg.stop_tet;
    int sms = 0;
    int per_sm = max_persistent_ctas(cfg.mode, false, cfg.bounded, cfg.block, &sms);
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
    int64_t grid = (int64_t)per_sm * sms;
    const int64_t need = (n + cfg.block - 1) / cfg.block;
    if (!n_dev && grid > need) grid = need;
    cudaError_t e = cfg.bounded
        ? dispatch<true, false>(cfg.mode, cfg.format, mv, rays, hits, nullptr, 0, W, cfg.block, (int)grid, cfg.events, s)
        : dispatch<false, false>(cfg.mode, cfg.format, mv, rays, hits, nullptr, 0, W, cfg.block, (int)grid, cfg.events, s);
    if (e != cudaSuccess) {
        tm_set_error("trace launch", e);
        cudaFreeAsync(cursor, s);
        return TM_ERR_CUDA;
    }
    tm_count_launches(3);
    TM_CUDA(cudaFreeAsync(cursor, s));
    return TM_OK;
}

tm_status launch_trace_batch(const BatchDesc *descs_dev, int n_meshes, int64_t total,
                             const TraceConfig &cfg, unsigned long long *cursor, cudaStream_t s,
                             bool count) {
    if (!valid_config(cfg) || n_meshes < 1 || n_meshes > kMaxBatch) return TM_ERR_ARG;
    if (total == 0) return TM_OK;
    WalkParams W;
    W.n_cap = total;
    W.n_dev = nullptr;
    W.cursor = cursor;
    W.max_steps = cfg.max_steps;
    W.tau_rel = cfg.tau;
    W.refill = cfg.refill;
    W.batch_steps = cfg.batch_steps;
    W.stop_tet = nullptr;
    int sms = 0;
    int per_sm = max_persistent_ctas(cfg.mode, true, false, cfg.block, &sms);
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
    int64_t grid = (int64_t)per_sm * sms;
    const int64_t need = (total + cfg.block - 1) / cfg.block;
    if (grid > need) grid = need;
    TM_CUDA(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s));
    MeshView dummy{};
    if (cfg.format == TM_FORMAT_TET20) return TM_ERR_ARG;
    cudaError_t e = dispatch<false, true>(cfg.mode, cfg.format, dummy, nullptr, nullptr, descs_dev,
                                          n_meshes, W, cfg.block, (int)grid, nullptr, s);
    if (e != cudaSuccess) {
        tm_set_error("trace (batch) launch", e);
        return TM_ERR_CUDA;
    }
    if (count) tm_count_launches(3);
    return TM_OK;
}
