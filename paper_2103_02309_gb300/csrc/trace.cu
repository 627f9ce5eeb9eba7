// Persistent ray traversal kernel (Sec. 4 and Sec. 7 of the paper) for sm_103a.
//
// One lane holds one ray in registers: its current tet, the tet it came
// from, the entry face (three vertex ids and their 2-D projections) and the
// scaled basis.  Each step (Alg. 6) reads one 16-byte Tet16 record and one
// 16-byte point, projects the new vertex (Eq. 3 with the projected origin),
// picks the exit slot with Alg. 1 and decodes the next tet from the xor
// neighbours (Alg. 7):
//   idx3 = idx0 ^ idx1 ^ idx2 ^ VX
//   ra = rank of idx3, rb = rank of idx_exit among the four vertex ids
//   N3 = ra == 3 ? prev : prev ^ NX_ra ;  next = rb == 3 ? N3 : N3 ^ NX_rb
// and stops at a flagged (constrained or boundary) neighbour.  Alg. 1 is
// evaluated from the three signs det(p3, p_k) without branches.
//
// Warps are persistent: lanes whose ray ended are refilled from a global
// cursor once `refill` lanes are idle (ballot + popc, one atomicAdd per
// warp, the new ray ids handed out by rank within the idle mask), so that
// the rays of one grab are consecutive and warps stay full as rays end after
// different numbers of steps (the persistent-threads scheme of Aila & Laine,
// "Understanding the efficiency of ray traversal on GPUs", HPG 2009).
#include <cmath>

#include "walk.cuh"

namespace tmk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxBatch = 64;

struct TraceParams {
    int64_t n_cap;
    const int64_t *n_dev;
    unsigned long long *cursor;
    uint32_t max_steps;
    float tau_rel;  // sign-test guard threshold relative to the mesh extent
    int refill;
    int batch_steps;
};

// Final hit in double precision: (t, b1, b2).  Out of line: the guard path.
__device__ __noinline__ static float4 mt_hit_fp64(const float4 o4, const float4 d4, const float4 a4,
                                                  const float4 b4, const float4 c4) {
    double t, u, v, cond;
    mt_hit<double>(o4, d4, a4, b4, c4, t, u, v, cond);
    return make_float4((float)t, (float)u, (float)v, 0.f);
}

// In guard mode the float32 ray-triangle test is redone in double precision
// when its condition estimate (see mt_hit) exceeds kFinalCond, i.e. when the
// float32 t could be off by more than about 2e-6 relative.
constexpr float kFinalCond = 32.f;

// Writes the hit (or miss) of a finished ray.  `code` is the flagged
// neighbour value that ended the walk in tet `tet`.
template <int MODE>
__device__ __forceinline__ void finish(const MeshView &mv, const tm_ray *rp, tm_hit *hp,
                                       uint32_t code, int32_t tet, uint32_t steps, uint32_t flags) {
    const float4 w0 = __ldg(reinterpret_cast<const float4 *>(rp));
    const float4 w1 = __ldg(reinterpret_cast<const float4 *>(rp) + 1);
    int32_t tri = -1, cf = -1;
    float t = __int_as_float(0x7f800000), b1 = 0.f, b2 = 0.f;
    if (code != TM_BOUNDARY && (int32_t)(code & ~TM_CFACE_FLAG) >= mv.nc) {
        flags |= TM_HIT_BAD_ID;
        code = TM_BOUNDARY;
    }
    if (code != TM_BOUNDARY) {
        const int32_t c = (int32_t)(code & ~TM_CFACE_FLAG);
        const int4 r0 = __ldg(mv.cface + 2 * c);
        const int4 r1 = __ldg(mv.cface + 2 * c + 1);  // vertex ids validated by the host build
        const float4 a = __ldg(mv.pts + r1.x), b = __ldg(mv.pts + r1.y), d = __ldg(mv.pts + r1.z);
        float th, u, v;
        if (MODE == FP64) {
            const float4 h = mt_hit_fp64(w0, w1, a, b, d);
            th = h.x; u = h.y; v = h.z;
        } else {
            float cond;
            mt_hit<float>(w0, w1, a, b, d, th, u, v, cond);
            if (MODE == FP32G && !(cond <= kFinalCond)) {
                const float4 h = mt_hit_fp64(w0, w1, a, b, d);
                th = h.x; u = h.y; v = h.z;
                flags |= TM_HIT_FINAL_FP64;
            }
        }
        if (th <= w1.w) {
            tri = r0.x;
            cf = c;
            t = th;
            b1 = u;
            b2 = v;
            if (r0.y != tet) flags |= TM_HIT_SIDE_NEG;
        }
    }
    __stcs(reinterpret_cast<int4 *>(hp), make_int4(tri, __float_as_int(t), __float_as_int(b1),
                                                   __float_as_int(b2)));
    __stcs(reinterpret_cast<int4 *>(hp) + 1, make_int4(tet, cf, (int)steps, (int)flags));
}

// Once per ray and with only value arguments: out of line by default.
#ifdef TM_FINISH_INLINE
#define TM_FINISH_ATTR __forceinline__
#else
#define TM_FINISH_ATTR __noinline__
#endif

template <int MODE>
__device__ TM_FINISH_ATTR void finish_ray(const MeshView mv, const tm_ray *rp, tm_hit *hp,
                                          uint32_t code, int32_t tet, uint32_t steps,
                                          uint32_t flags) {
    finish<MODE>(mv, rp, hp, code, tet, steps, flags);
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

template <class R, bool BOUNDED> struct Depth {
    __device__ __forceinline__ void init(R, R, R, R, R, R, float) {}
    __device__ __forceinline__ void set(int, const float4 &) {}
    __device__ __forceinline__ bool beyond() const { return false; }
};
template <class R> struct Depth<R, true> {
    R dx, dy, dz, dod, zmax, z0, z1, z2;
    __device__ __forceinline__ void init(R ox, R oy, R oz, R x, R y, R z, float tmax) {
        dx = x; dy = y; dz = z;
        dod = rfma(dz, oz, rfma(dy, oy, rmul(dx, ox)));
        zmax = R(tmax) * rfma(dz, dz, rfma(dy, dy, rmul(dx, dx)));
    }
    __device__ __forceinline__ R depth(const float4 &p) const {
        return rfma(dz, R(p.z), rfma(dy, R(p.y), rmul(dx, R(p.x)))) - dod;
    }
    __device__ __forceinline__ void set(int slot, const float4 &p) {
        const R z = depth(p);
        if (slot == 0) z0 = z; else if (slot == 1) z1 = z; else z2 = z;
    }
    // the entry face of the next tet lies entirely beyond t_max
    __device__ __forceinline__ bool beyond() const { return fmin(z0, fmin(z1, z2)) > zmax; }
};

// Starts the ray at rp: basis, projected origin, and the exit face of its
// start tet (interior start) or of the tet behind its restart face.  Returns
// true when the walk continues in S.tet; otherwise the hit is written.
template <int MODE, bool BOUNDED>
__device__ __forceinline__ bool start_ray(const MeshView &mv, const tm_ray *rp, tm_hit *hp,
                                          WalkState<typename RealOf<MODE>::T> &S,
                                          Basis<typename RealOf<MODE>::T> &B,
                                          Depth<typename RealOf<MODE>::T, BOUNDED> &Z,
                                          SignCtx &sc, uint32_t &steps) {
    typedef typename RealOf<MODE>::T R;
    const float4 w0 = __ldcs(reinterpret_cast<const float4 *>(rp));
    const float4 w1 = __ldcs(reinterpret_cast<const float4 *>(rp) + 1);
    B = make_basis<R>(R(w1.x), R(w1.y), R(w1.z), R(w0.x), R(w0.y), R(w0.z));
    sc.flags = 0;
    steps = 0;
    const int32_t start = __float_as_int(w0.w);
    uint32_t next = TM_BOUNDARY;
    int32_t T = -1;
    bool ok = false;
    if (start >= 0) {
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
        if (c < mv.nc) {
            const int4 r0 = __ldg(mv.cface + 2 * c);
            T = (code & 1) ? r0.z : r0.y;
        }
        if (T >= mv.nt) T = -1;
        if (T >= 0) {
            const int4 cn = __ldg(mv.cold + 2 * T + 1);
            const uint32_t want = TM_CFACE_FLAG | (uint32_t)c;
            int skip = (uint32_t)cn.x == want ? 0 : (uint32_t)cn.y == want ? 1
                     : (uint32_t)cn.z == want ? 2 : (uint32_t)cn.w == want ? 3 : -1;
            if (skip >= 0) {
                ok = line_init<MODE>(mv, B, T, skip, sc, S, next);
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
    if (!ok) {
        finish_ray<MODE>(mv, rp, hp, TM_BOUNDARY, T, steps, sc.flags | TM_HIT_BAD_START);
        return false;
    }
    if (next & TM_CFACE_FLAG) {
        finish_ray<MODE>(mv, rp, hp, next, S.prev, steps, sc.flags);
        return false;
    }
    S.tet = (int32_t)next;
    if (BOUNDED) {
        Z.init(R(w0.x), R(w0.y), R(w0.z), R(w1.x), R(w1.y), R(w1.z), w1.w);
        Z.set(0, __ldg(mv.pts + S.i0));
        Z.set(1, __ldg(mv.pts + S.i1));
        Z.set(2, __ldg(mv.pts + S.i2));
        if (Z.beyond()) {
            finish_ray<MODE>(mv, rp, hp, TM_BOUNDARY, S.prev, steps, sc.flags);
            return false;
        }
    }
    return true;
}

// Register budget per thread of the walk (FP32 arms; the FP64 arm needs
// double-width state).  Set by measurement on GB300.
#ifndef TM_TRACE_MAXREG
#define TM_TRACE_MAXREG 64
#endif
#ifndef TM_TRACE_MAXREG_FP64
#define TM_TRACE_MAXREG_FP64 80
#endif

template <int MODE, bool BOUNDED, bool MULTI>
__global__ void __maxnreg__(MODE == FP64 ? TM_TRACE_MAXREG_FP64 : TM_TRACE_MAXREG)
trace_kernel(const __grid_constant__ MeshView mv0, const tm_ray *__restrict__ rays0,
             tm_hit *__restrict__ hits0, const BatchDesc *__restrict__ descs, int n_meshes,
             const __grid_constant__ TraceParams P) {
    typedef typename RealOf<MODE>::T R;
    extern __shared__ BatchDesc sdesc[];
    if (MULTI) {
        for (int i = threadIdx.x; i < n_meshes; i += blockDim.x) sdesc[i] = descs[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    int64_t n = P.n_cap;
    if (P.n_dev) n = min(n, *P.n_dev);

    bool active = false, pool_empty = false;
    int32_t m = 0, local = 0;
    const int4 *tet16 = mv0.tet16;
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

    for (;;) {
        const unsigned idle = __ballot_sync(kFull, !active);
        const int n_idle = __popc(idle);
        if (!pool_empty && n_idle >= P.refill) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(P.cursor, (unsigned long long)n_idle);
            base = __shfl_sync(kFull, base, 0);
            if (base + (unsigned long long)n_idle >= (unsigned long long)n) pool_empty = true;
            const unsigned long long r = base + __popc(idle & ((1u << lane) - 1u));
            if (!active && r < (unsigned long long)n) {
                tm_hit *hp;
                if (MULTI) {
                    int lo = 0, hi = n_meshes - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if ((unsigned long long)sdesc[mid].offset <= r) lo = mid; else hi = mid - 1;
                    }
                    m = lo;
                    local = (int32_t)(r - (unsigned long long)sdesc[m].offset);
                    if (sdesc[m].perm) local = sdesc[m].perm[local];
                    tet16 = sdesc[m].mesh.tet16;
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
                active = start_ray<MODE, BOUNDED>(MULTI ? sdesc[m].mesh : mv0, sc.ray, hp, S, B, Z,
                                                  sc, steps);
            }
        }
        if (!__any_sync(kFull, active)) {
            if (pool_empty) break;
            continue;
        }
        for (int k = 0; k < P.batch_steps; ++k) {
            if (!active) continue;
            // ---- one step of Alg. 6 / Alg. 7 ----
            const int4 rec = __ldg(tet16 + S.tet);
            const int32_t i3 = S.i0 ^ S.i1 ^ S.i2 ^ rec.x;
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
                const int e = exit_slot_bits(step_signs<MODE>(S, p3, i3, m3, sc));
                const int ra = (S.i0 < i3) + (S.i1 < i3) + (S.i2 < i3);
                const int32_t ie = e == 0 ? S.i0 : (e == 1 ? S.i1 : S.i2);
                const int rb = (S.i0 < ie) + (S.i1 < ie) + (S.i2 < ie) + (i3 < ie);
                const uint32_t nxa = ra == 0 ? rec.y : (ra == 1 ? rec.z : (ra == 2 ? rec.w : 0));
                const uint32_t nxb = rb == 0 ? rec.y : (rb == 1 ? rec.z : (rb == 2 ? rec.w : 0));
                const uint32_t next = (uint32_t)S.prev ^ nxa ^ nxb;
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
                } else if (BOUNDED && Z.beyond()) {
                    done = true;
                    code = TM_BOUNDARY;
                } else {
                    S.prev = S.tet;
                    S.tet = (int32_t)next;
                }
            }
            if (done) {
                finish_ray<MODE>(MULTI ? sdesc[m].mesh : mv0, sc.ray,
                                 MULTI ? sdesc[m].hits + local : hits0 + local, code, S.tet, steps,
                                 sc.flags);
                active = false;
            }
        }
    }
}

}  // namespace tmk

using namespace tmk;

namespace {

template <int MODE, bool BOUNDED, bool MULTI>
cudaError_t launch_one(const MeshView &mv, const tm_ray *rays, tm_hit *hits, const BatchDesc *descs,
                       int n_meshes, const TraceParams &P, int block, int grid, cudaStream_t s) {
    const size_t smem = MULTI ? sizeof(BatchDesc) * (size_t)n_meshes : 0;
    trace_kernel<MODE, BOUNDED, MULTI><<<grid, block, smem, s>>>(mv, rays, hits, descs, n_meshes, P);
    return cudaGetLastError();
}

template <int MODE, bool BOUNDED, bool MULTI>
int occupancy(int block, size_t smem) {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, trace_kernel<MODE, BOUNDED, MULTI>, block, smem);
    return nb;
}

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

template <bool BOUNDED, bool MULTI>
int occupancy_mode(int mode, int block, size_t smem) {
    switch (mode) {
        case FP32G: return occupancy<FP32G, BOUNDED, MULTI>(block, smem);
        case FP32: return occupancy<FP32, BOUNDED, MULTI>(block, smem);
        default: return occupancy<FP64, BOUNDED, MULTI>(block, smem);
    }
}

template <bool BOUNDED, bool MULTI>
cudaError_t dispatch(int mode, const MeshView &mv, const tm_ray *rays, tm_hit *hits,
                     const BatchDesc *descs, int n_meshes, const TraceParams &P, int block, int grid,
                     cudaStream_t s) {
    switch (mode) {
        case FP32G: return launch_one<FP32G, BOUNDED, MULTI>(mv, rays, hits, descs, n_meshes, P, block, grid, s);
        case FP32: return launch_one<FP32, BOUNDED, MULTI>(mv, rays, hits, descs, n_meshes, P, block, grid, s);
        default: return launch_one<FP64, BOUNDED, MULTI>(mv, rays, hits, descs, n_meshes, P, block, grid, s);
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
    c.block = (o && o->block) ? o->block : 512;
    c.refill = (o && o->refill) ? o->refill : 8;
    c.batch_steps = (o && o->batch_steps) ? o->batch_steps : 16;
    c.ctas_per_sm = o ? o->ctas_per_sm : 0;
    c.bounded = o ? o->tmax_early_exit != 0 : false;
    return c;
}

static bool valid_config(const TraceConfig &c) {
    return (c.mode == FP32G || c.mode == FP32 || c.mode == FP64) && c.block >= 32 &&
           c.block <= 1024 && c.block % 32 == 0 && c.refill >= 1 && c.refill <= 32 &&
           c.batch_steps >= 1 && c.batch_steps <= 256 && c.ctas_per_sm >= 0;
}

tm_status launch_trace(const MeshView &mv, const tm_ray *rays, int64_t n, const int64_t *n_dev,
                       tm_hit *hits, const TraceConfig &cfg, cudaStream_t s) {
    if (!valid_config(cfg)) return TM_ERR_ARG;
    if (n == 0) return TM_OK;
    if (n > INT32_MAX) return TM_ERR_TOO_LARGE;
    unsigned long long *cursor = nullptr;
    TM_CUDA(cudaMallocAsync((void **)&cursor, sizeof(unsigned long long), s));
    TM_CUDA(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s));
    TraceParams P;
    P.n_cap = n;
    P.n_dev = n_dev;
    P.cursor = cursor;
    P.max_steps = cfg.max_steps;
    P.tau_rel = cfg.tau;
    P.refill = cfg.refill;
    P.batch_steps = cfg.batch_steps;
    int sms = 0;
    const bool bnd = cfg.bounded;
    const int mode = cfg.mode;
    int per_sm = max_persistent_ctas(mode, false, bnd, cfg.block, &sms);
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
    int64_t grid = (int64_t)per_sm * sms;
    const int64_t need = (n + cfg.block - 1) / cfg.block;
    if (!n_dev && grid > need) grid = need;
    cudaError_t e = bnd ? dispatch<true, false>(mode, mv, rays, hits, nullptr, 0, P, cfg.block, (int)grid, s)
                        : dispatch<false, false>(mode, mv, rays, hits, nullptr, 0, P, cfg.block, (int)grid, s);
    if (e != cudaSuccess) {
        tm_set_error("trace_kernel launch", e);
        cudaFreeAsync(cursor, s);
        return TM_ERR_CUDA;
    }
    tm_count_launches(1);
    TM_CUDA(cudaFreeAsync(cursor, s));
    return TM_OK;
}

tm_status launch_trace_batch(const BatchDesc *descs_dev, int n_meshes, int64_t total,
                             const TraceConfig &cfg, unsigned long long *cursor, cudaStream_t s,
                             bool count) {
    if (!valid_config(cfg) || n_meshes < 1 || n_meshes > kMaxBatch) return TM_ERR_ARG;
    if (total == 0) return TM_OK;
    TraceParams P;
    P.n_cap = total;
    P.n_dev = nullptr;
    P.cursor = cursor;
    P.max_steps = cfg.max_steps;
    P.tau_rel = cfg.tau;
    P.refill = cfg.refill;
    P.batch_steps = cfg.batch_steps;
    int sms = 0;
    const int mode = cfg.mode;
    int per_sm = max_persistent_ctas(mode, true, false, cfg.block, &sms);
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
    int64_t grid = (int64_t)per_sm * sms;
    const int64_t need = (total + cfg.block - 1) / cfg.block;
    if (grid > need) grid = need;
    TM_CUDA(cudaMemsetAsync(cursor, 0, sizeof(unsigned long long), s));
    MeshView dummy{};
    cudaError_t e = dispatch<false, true>(mode, dummy, nullptr, nullptr, descs_dev, n_meshes, P,
                                          cfg.block, (int)grid, s);
    if (e != cudaSuccess) {
        tm_set_error("trace_kernel (batch) launch", e);
        return TM_ERR_CUDA;
    }
    if (count) tm_count_launches(1);
    return TM_OK;
}
