// Ray generation on the device: primary pinhole rays in warp tiles, and
// rays restarted from hit faces (Sec. 6 of the paper): diffuse bounce /
// ambient occlusion and reflection into the arrival-side tet, refraction
// into the tet across the face, shadow rays into the side facing a point
// light.  Rays from hits are compacted with a three-pass scan (count per
// block, scan of the block counts, emit), so the output order does not
// depend on scheduling: shadow and specular rays in hit order, diffuse and
// occlusion rays by length bucket; within a bucket, by block of 1024 hits,
// then by the octant of the hit's first direction, then in hit order.
#include <mutex>
#include <string>

#include "tm_internal.h"

namespace tmk {

constexpr int kTileW = 8, kTileH = 4;

// A 32-byte ray written by one 256-bit streaming store (sm_100 and later;
// the C ABI requires 32-byte aligned ray buffers) instead of two 128-bit
// ones, so that L2 never receives a sector in halves.
#ifndef TM_ST256
#define TM_ST256 1
#endif
__device__ __forceinline__ void store32_cs(void *p, const float4 &a, const float4 &b) {
    const unsigned long long q0 = ((unsigned long long)__float_as_uint(a.y) << 32) | __float_as_uint(a.x);
    const unsigned long long q1 = ((unsigned long long)__float_as_uint(a.w) << 32) | __float_as_uint(a.z);
    const unsigned long long q2 = ((unsigned long long)__float_as_uint(b.y) << 32) | __float_as_uint(b.x);
    const unsigned long long q3 = ((unsigned long long)__float_as_uint(b.w) << 32) | __float_as_uint(b.z);
    asm volatile("st.global.cs.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(q0), "l"(q1), "l"(q2), "l"(q3)
                 : "memory");
}

// One warp per 8x4 pixel tile (lane -> column lane % 8, row lane / 8), a
// block's eight warps along a tile row, blockIdx.y the tile row: the ray
// index follows from the pixel with shifts and products only.  Tile rows
// hold kTileH full rows (the last may be shorter); within a row, tiles are
// kTileW wide (the last may be narrower), and a tile's rays are row-major.
__global__ void __launch_bounds__(256)
gen_primary_kernel(const __grid_constant__ tm_camera cam, const int32_t *__restrict__ start,
                   float tmax, tm_ray *__restrict__ rays) {
    const int64_t W = cam.width, H = cam.height;
    const int64_t tiles_x = (W + kTileW - 1) / kTileW, tiles_y = (H + kTileH - 1) / kTileH;
    const int32_t st = *start;
    const int lane = threadIdx.x & 31;
    const int64_t tx = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (tx >= tiles_x) return;
    const int64_t lx = lane % kTileW, ly = lane / kTileW;
    const int64_t tw = min((int64_t)kTileW, W - tx * kTileW);
    for (int64_t ty = blockIdx.y; ty < tiles_y; ty += gridDim.y) {
        const int64_t th = min((int64_t)kTileH, H - ty * kTileH);
        if (lx >= tw || ly >= th) continue;
        const int64_t px = tx * kTileW + lx, py = ty * kTileH + ly;
        const int64_t r = ty * kTileH * W + tx * kTileW * th + ly * tw + lx;
        const float sx = __fmul_rn(__fsub_rn(__fmul_rn(__fadd_rn((float)px, 0.5f), cam.kx), 1.0f), cam.tx);
        const float sy = __fmul_rn(__fsub_rn(1.0f, __fmul_rn(__fadd_rn((float)py, 0.5f), cam.ky)), cam.ty);
        const float s2 = __fadd_rn(__fadd_rn(__fmul_rn(sx, sx), __fmul_rn(sy, sy)), 1.0f);
        const float L = __fsqrt_rn(s2);
        const float dx = __fdiv_rn(sx, L), dy = __fdiv_rn(sy, L), dz = __fdiv_rn(1.0f, L);
#if TM_ST256
        store32_cs(rays + r, make_float4(cam.eye[0], cam.eye[1], cam.eye[2], __int_as_float(st)),
                   make_float4(dx, dy, dz, tmax));
#else
        float4 *out = reinterpret_cast<float4 *>(rays + r);
        __stcs(out, make_float4(cam.eye[0], cam.eye[1], cam.eye[2], __int_as_float(st)));
        __stcs(out + 1, make_float4(dx, dy, dz, tmax));
#endif
    }
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based
// generator: draw i of stream `seed` is mix64(seed + (i+1) * golden gamma).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float uniform24(uint64_t seed, uint64_t i) {
    const uint64_t z = mix64(seed + (i + 1ull) * 0x9E3779B97F4A7C15ull);
    return (float)(z >> 40) * (1.0f / 16777216.0f);
}

constexpr int kScanBlock = 1024;

__device__ __forceinline__ int64_t valid_count(int64_t n, const int64_t *n_dev) {
    return n_dev ? min(n, *n_dev) : n;
}

// A hit the generators use: a triangle id, on a constrained face of this
// mesh (a foreign or corrupted record counts as a miss, never as an index).
__device__ __forceinline__ bool usable_hit(int32_t tri, int32_t cface, int32_t nc) {
    return tri >= 0 && (uint32_t)cface < (uint32_t)nc;
}

__global__ void __launch_bounds__(kScanBlock)
count_hits_kernel(const tm_hit *__restrict__ hits, int64_t n, const int64_t *n_dev, int32_t nc,
                  int32_t *__restrict__ block_counts) {
    const int64_t nv = valid_count(n, n_dev);
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    const bool hit = i < nv && usable_hit(__ldg(&hits[i].tri), __ldg(&hits[i].cface), nc);
    const int c = __syncthreads_count(hit);
    if (threadIdx.x == 0) block_counts[blockIdx.x] = c;
}

// Exclusive scan of the block counts in one block; total at offsets[nb].
// Each warp takes a contiguous segment of the counts and reads it 32 at a
// time (one coalesced line per read): first the segment's sum, then, after
// the block has scanned the 32 warp sums, the offsets, with a warp scan per
// line and a running carry.  One pass for any number of counts (the diffuse
// generator has one per block and length bucket).
__global__ void __launch_bounds__(kScanBlock)
scan_counts_kernel(const int32_t *__restrict__ counts, int64_t nb, int64_t *__restrict__ offsets,
                   int per_hit, int64_t *__restrict__ count_out) {
    constexpr int kWarps = kScanBlock / 32;
    __shared__ int64_t warp_base[kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t seg = (nb + kWarps - 1) / kWarps;
    const int64_t lo = min(nb, warp * seg), hi = min(nb, lo + seg);
    int64_t v = 0;
#pragma unroll 8
    for (int64_t i = lo + lane; i < hi; i += 32) v += __ldcg(counts + i);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) warp_base[warp] = v;
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the warp sums
        const int64_t w = warp_base[lane];
        int64_t x = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        warp_base[lane] = x - w;
        if (lane == 31) {
            offsets[nb] = x;
            *count_out = x * per_hit;
        }
    }
    __syncthreads();
    // kLines lines of counts are read before the first is scanned, so the
    // reads' latency is paid once per kLines lines, not once per line; a
    // line's sum (32 block counts of at most kScanBlock) fits in 32 bits
    constexpr int kLines = 8;
    int64_t carry = warp_base[warp];
    for (int64_t base = lo; base < hi; base += 32 * kLines) {
        int c[kLines];
#pragma unroll
        for (int u = 0; u < kLines; ++u) {
            const int64_t i = base + 32 * u + lane;
            c[u] = i < hi ? __ldcg(counts + i) : 0;
        }
#pragma unroll
        for (int u = 0; u < kLines; ++u) {
            const int64_t i = base + 32 * u + lane;
            int x = c[u];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (i < hi) offsets[i] = carry + (x - c[u]);
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    }
}

// One hit of the launch, read by the emit kernels.
struct HitIn {
    int4 h0, h1;
    bool hit;
};
__device__ __forceinline__ HitIn load_hit(const tm_hit *hits, int64_t i, int64_t nv, int32_t nc) {
    HitIn r;
    r.h0 = make_int4(-1, 0, 0, 0);
    r.h1 = make_int4(0, 0, 0, 0);
    if (i < nv) {
        r.h0 = __ldcs(reinterpret_cast<const int4 *>(hits + i));
        r.h1 = __ldcs(reinterpret_cast<const int4 *>(hits + i) + 1);
    }
    r.hit = usable_hit(r.h0.x, r.h1.y, nc);
    return r;
}

// Output position of this thread's hit: the block's offset from the scan
// plus the hits of the lower threads of the block.  Every thread of the
// block calls it.
__device__ __forceinline__ int64_t hit_position(bool hit, const int64_t *offsets) {
    __shared__ int warp_counts[kScanBlock / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, hit);
    if (lane == 0) warp_counts[warp] = __popc(bal);
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += warp_counts[w];
    before += __popc(bal & ((1u << lane) - 1u));
    return offsets[blockIdx.x] + before;
}

// The hit point x = a + b1 (b - a) + b2 (c - a) on triangle (a, b, c) (input
// vertex order) and the unnormalised normal (b - a) x (c - a).
struct HitGeom {
    float ox, oy, oz;
    float nx, ny, nz;
    float4 a;
};
__device__ __forceinline__ HitGeom hit_geometry(const MeshView &mv, const HitIn &h) {
    HitGeom g;
    const int32_t c = h.h1.y;
    const int4 g0 = __ldg(mv.cgeo + 3 * c), g1 = __ldg(mv.cgeo + 3 * c + 1),
               g2 = __ldg(mv.cgeo + 3 * c + 2);
    const float4 a = make_float4(__int_as_float(g0.x), __int_as_float(g0.y), __int_as_float(g0.z), 0.f);
    const float4 b = make_float4(__int_as_float(g1.x), __int_as_float(g1.y), __int_as_float(g1.z), 0.f);
    const float4 d = make_float4(__int_as_float(g2.x), __int_as_float(g2.y), __int_as_float(g2.z), 0.f);
    const float b1 = __int_as_float(h.h0.z), b2 = __int_as_float(h.h0.w);
    const float e1x = b.x - a.x, e1y = b.y - a.y, e1z = b.z - a.z;
    const float e2x = d.x - a.x, e2y = d.y - a.y, e2z = d.z - a.z;
    g.ox = a.x + b1 * e1x + b2 * e2x;
    g.oy = a.y + b1 * e1y + b2 * e2y;
    g.oz = a.z + b1 * e1z + b2 * e2z;
    g.nx = e1y * e2z - e1z * e2y;
    g.ny = e1z * e2x - e1x * e2z;
    g.nz = e1x * e2y - e1y * e2x;
    g.a = a;
    return g;
}

__device__ __forceinline__ void put_ray(tm_ray *out, int64_t o, float ox, float oy, float oz,
                                        int32_t start, float dx, float dy, float dz, float tmax) {
#if TM_ST256
    store32_cs(out + o, make_float4(ox, oy, oz, __int_as_float(start)), make_float4(dx, dy, dz, tmax));
#else
    float4 *r = reinterpret_cast<float4 *>(out + o);
    __stcs(r, make_float4(ox, oy, oz, __int_as_float(start)));
    __stcs(r + 1, make_float4(dx, dy, dz, tmax));
#endif
}

// Cosine-weighted directions about the normal of a hit, turned toward its
// arrival side, in an orthonormal frame (Duff et al., JCGT 2017).
struct BounceFrame {
    float ox, oy, oz;                      // the hit point
    float nx, ny, nz, t1x, t1y, t1z, t2x, t2y, t2z;
    int32_t start;                         // restart code of the hit face's arrival side
};
__device__ __forceinline__ BounceFrame bounce_frame(const MeshView &mv, const HitIn &h) {
    BounceFrame f;
    const int32_t c = h.h1.y;
    const int side = (h.h1.w & TM_HIT_SIDE_NEG) ? 1 : 0;
    const HitGeom g = hit_geometry(mv, h);
    f.ox = g.ox; f.oy = g.oy; f.oz = g.oz;
    float nx = g.nx, ny = g.ny, nz = g.nz;
    const float inv = rsqrtf(nx * nx + ny * ny + nz * nz) * (side ? -1.f : 1.f);
    nx *= inv; ny *= inv; nz *= inv;
    const float sgn = nz >= 0.f ? 1.f : -1.f;
    const float aa = -1.f / (sgn + nz), bb = nx * ny * aa;
    f.nx = nx; f.ny = ny; f.nz = nz;
    f.t1x = 1.f + sgn * nx * nx * aa; f.t1y = sgn * bb; f.t1z = -sgn * nx;
    f.t2x = bb; f.t2y = sgn + ny * ny * aa; f.t2z = -ny;
    f.start = -1 - (2 * c + side);
    return f;
}
// The hardware's approximate square root (relative error near 2^-23;
// +0 at +0).
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
// Direction k of hit i: draws 2 (i per_hit + k) and 2 (i per_hit + k) + 1.
__device__ __forceinline__ float3 bounce_dir(const BounceFrame &f, uint64_t seed, int64_t i, int per_hit,
                                             int k) {
    const uint64_t cnt = 2ull * ((uint64_t)i * (uint64_t)per_hit + (uint64_t)k);
    const float u0 = uniform24(seed, cnt), u1 = uniform24(seed, cnt + 1);
    // phi = 2 pi u0 = psi + pi with psi = 2 pi (u0 - 1/2) in [-pi, pi), the
    // range of the fast sine and cosine (absolute error about 5e-7 there):
    // sin phi = -sin psi, cos phi = -cos psi
    float sp, cp;
    __sincosf(6.283185307f * (u0 - 0.5f), &sp, &cp);
    sp = -sp;
    cp = -cp;
    const float s = sqrt_approx(u1), lz = sqrt_approx(fmaxf(0.f, 1.f - u1));
    float dx = s * cp * f.t1x + s * sp * f.t2x + lz * f.nx;
    float dy = s * cp * f.t1y + s * sp * f.t2y + lz * f.ny;
    float dz = s * cp * f.t1z + s * sp * f.t2z + lz * f.nz;
    const float il = rsqrtf(dx * dx + dy * dy + dz * dz);
    return make_float3(dx * il, dy * il, dz * il);
}

// Length bucket of a hit's rays, from its first ray: 0 when the longest
// walk that ray can make (to the mesh's bounding box, or to t_max) spans
// the box, up to kLengthBuckets - 1 when it ends next to the origin.  A
// persistent walk ends with a tail: once its ray pool is empty a few long
// rays keep a few lanes busy, and a long ray taken late sets the tail's
// length.  Diffuse bounce rays are spread out in length, so the generator
// writes them bucket by bucket, farthest first, and a walk over them takes
// the long ones early.  Measured on GB300 on the precision workload's bounce
// rays, ordered on the host: 2 buckets cut their walk by 13 %, 4 by 16 %, a
// full sort by that distance by 19 %, with slower start and finish phases.
constexpr int kLengthBuckets = 8;
__device__ __forceinline__ int length_bucket(const MeshView &mv, float ox, float oy, float oz,
                                             const float3 &d, float tmax) {
    float t = tmax;
    const float ov[3] = {ox, oy, oz}, dv[3] = {d.x, d.y, d.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // the bucket only orders the rays: a fast quotient (2 ulp) will do
        if (dv[a] > 0.f) t = fminf(t, __fdividef(mv.hi[a] - ov[a], dv[a]));
        else if (dv[a] < 0.f) t = fminf(t, __fdividef(mv.lo[a] - ov[a], dv[a]));
    }
    const float len = t / fmaxf(mv.extent, 1e-30f);   // d has unit length
    if (!(len < 1.f)) return 0;                        // also NaN
    const int b = (int)((1.f - fmaxf(len, 0.f)) * (float)kLengthBuckets);
    return b < kLengthBuckets ? b : kLengthBuckets - 1;
}

// The diffuse / occlusion generator's count pass runs kCountThreads threads
// a block and its emit pass kEmitThreads; each thread takes PER = kScanBlock
// / THREADS hits of the block's kScanBlock (hit base + j * THREADS + thread
// for j = 0 .. PER-1, so every load is coalesced).  A thread issues the reads
// of all its hits before it waits on any, and then the reads of their
// triangles, instead of waiting on two dependent reads per hit.  Within a
// block, hit order is (j, thread).  The emit pass holds more per hit, so it
// takes fewer hits a thread and keeps more warps.
constexpr int kCountThreads = 256;
constexpr int kEmitThreads = 512;

// Frames and buckets of this thread's hits (-1: no usable hit).
template <int PER> struct GenHits {
    HitIn h[PER];
    BounceFrame f[PER];
    float3 d0[PER];
    int b[PER];
};
template <int THREADS, int PER>
__device__ __forceinline__ void gen_hits(const MeshView &mv, const tm_hit *hits, int64_t n,
                                         const int64_t *n_dev, int per_hit, float tmax,
                                         uint64_t seed, GenHits<PER> &g) {
    const int64_t nv = valid_count(n, n_dev);
    const int64_t base = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
#pragma unroll
    for (int j = 0; j < PER; ++j) g.h[j] = load_hit(hits, base + j * THREADS, nv, mv.nc);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        g.b[j] = -1;
        if (g.h[j].hit) {
            g.f[j] = bounce_frame(mv, g.h[j]);
            g.d0[j] = bounce_dir(g.f[j], seed, base + j * THREADS, per_hit, 0);
            g.b[j] = length_bucket(mv, g.f[j].ox, g.f[j].oy, g.f[j].oz, g.d0[j], tmax);
        }
    }
}

// Per warp and j, the hits of each bucket (ballots); every thread calls it.
template <int THREADS, int PER>
__device__ __forceinline__ void gen_ballots(const int (&b)[PER], int (*wc)[kLengthBuckets][THREADS / 32],
                                            unsigned (&mine)[PER]) {
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        mine[j] = 0;
#pragma unroll
        for (int k = 0; k < kLengthBuckets; ++k) {
            const unsigned m = __ballot_sync(0xffffffffu, b[j] == k);
            if (b[j] == k) mine[j] = m;
            if (lane == 0) wc[j][k][warp] = __popc(m);
        }
    }
}

// Pass 1: counts[b * gridDim.x + block] = hits of the block in length
// bucket b (a scan of the counts in that order gives every bucket's blocks
// their place, bucket after bucket).
__global__ void __launch_bounds__(kCountThreads)
count_secondary_kernel(const __grid_constant__ MeshView mv, const tm_hit *__restrict__ hits,
                       int64_t n, const int64_t *n_dev, int per_hit, float tmax, uint64_t seed,
                       int32_t *__restrict__ counts) {
    constexpr int PER = kScanBlock / kCountThreads;
    __shared__ int wc[PER][kLengthBuckets][kCountThreads / 32];
    GenHits<PER> g;
    gen_hits<kCountThreads, PER>(mv, hits, n, n_dev, per_hit, tmax, seed, g);
    unsigned mine[PER];
    gen_ballots<kCountThreads, PER>(g.b, wc, mine);
    __syncthreads();
    if (threadIdx.x < kLengthBuckets) {
        int c = 0;
        for (int j = 0; j < PER; ++j)
            for (int w = 0; w < kCountThreads / 32; ++w) c += wc[j][threadIdx.x][w];
        counts[(int64_t)threadIdx.x * gridDim.x + blockIdx.x] = c;
    }
}

// Inside a block's share of a length group, hits go by the octant of their
// first ray's direction, then in hit order: keys b * 8 + octant, a warp's
// lanes of one key found with __match_any_sync, and one exclusive scan per
// group over (octant, j, warp).  Rays that leave a neighbourhood in one
// octant walk it together: on GB300 the precision workload's bounce walk
// took 1.5 % less time (0.4 % a step, the emit pass's extra work included).
#ifndef TM_EMIT_OCTANTS
#define TM_EMIT_OCTANTS 1
#endif
__global__ void __launch_bounds__(kEmitThreads, 2)
emit_secondary_kernel(const __grid_constant__ MeshView mv, const tm_hit *__restrict__ hits,
                      int64_t n, const int64_t *n_dev, const int64_t *__restrict__ offsets,
                      int per_hit, float tmax, uint64_t seed, tm_ray *__restrict__ out,
                      int32_t *__restrict__ src) {
    constexpr int PER = kScanBlock / kEmitThreads;
    constexpr int kWarps = kEmitThreads / 32;
    static_assert(PER * kWarps == 32, "one count a lane");
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    GenHits<PER> g;
    gen_hits<kEmitThreads, PER>(mv, hits, n, n_dev, per_hit, tmax, seed, g);
    unsigned mine[PER];
    int key[PER];
#if TM_EMIT_OCTANTS
    constexpr int kKeys = kLengthBuckets * 8;
    static_assert(kLengthBuckets * 2 == kWarps && kKeys * PER * kWarps == 256 * kLengthBuckets,
                  "two warps scan a group's 256 counts, four a thread");
    __shared__ __align__(16) int wk[kKeys][PER][kWarps];   // key-major: a group's counts are contiguous
    __shared__ int wtot[kWarps];
    for (int q = threadIdx.x; q < kKeys * PER * kWarps / 4; q += kEmitThreads)
        reinterpret_cast<int4 *>(&wk[0][0][0])[q] = make_int4(0, 0, 0, 0);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        key[j] = -1;
        if (g.b[j] >= 0)
            key[j] = g.b[j] * 8 + ((g.d0[j].x < 0.f) | ((g.d0[j].y < 0.f) << 1) | ((g.d0[j].z < 0.f) << 2));
        mine[j] = __match_any_sync(0xffffffffu, key[j]);
        if (key[j] >= 0 && lane == (unsigned)(__ffs(mine[j]) - 1)) wk[key[j]][j][warp] = __popc(mine[j]);
    }
    __syncthreads();
    {
        // group b = warp / 2: its 256 counts in (octant, j, warp) order, four
        // a thread; exclusive prefix left in place
        const int b = (int)(warp >> 1), t = (int)(((warp & 1u) << 5) | lane);
        int4 *cell = reinterpret_cast<int4 *>(&wk[b * 8][0][0]) + t;
        const int4 v = *cell;
        const int tot = v.x + v.y + v.z + v.w;
        int x = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        if (lane == 31) wtot[warp] = x;
        __syncthreads();
        int e = ((warp & 1u) ? wtot[warp - 1] : 0) + x - tot;
        int4 r;
        r.x = e; e += v.x;
        r.y = e; e += v.y;
        r.z = e; e += v.z;
        r.w = e;
        *cell = r;
    }
    __syncthreads();
#else
    __shared__ int wc[PER][kLengthBuckets][kEmitThreads / 32];
    gen_ballots<kEmitThreads, PER>(g.b, wc, mine);
    __syncthreads();
    // The block's hits of bucket b before (j, warp), in its hit order (j
    // first, then warp): warp b scans bucket b's PER x warps counts, one a
    // lane, and leaves the exclusive prefix in place.
    if (warp < (unsigned)kLengthBuckets) {
        int *cell = &wc[lane / kWarps][warp][lane % kWarps];
        const int v = *cell;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        *cell = x - v;
    }
    __syncthreads();
#endif
    const int64_t base = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int b = g.b[j];
        if (b < 0) continue;
        // the block's earlier hits of bucket b (and octant): those before
        // (j, warp), then the earlier lanes of this warp
#if TM_EMIT_OCTANTS
        const int before = wk[key[j]][j][warp] + __popc(mine[j] & ((1u << lane) - 1u));
#else
        (void)key;
        const int before = wc[j][b][warp] + __popc(mine[j] & ((1u << lane) - 1u));
#endif
        const int64_t pos = offsets[(int64_t)b * gridDim.x + blockIdx.x] + before;
        const int64_t i = base + j * kEmitThreads;
        const BounceFrame &f = g.f[j];
        for (int k = 0; k < per_hit; ++k) {
            const float3 d = k == 0 ? g.d0[j] : bounce_dir(f, seed, i, per_hit, k);
            const int64_t o = pos * per_hit + k;
            put_ray(out, o, f.ox, f.oy, f.oz, f.start, d.x, d.y, d.z, tmax);
            if (src) src[o] = (int32_t)i;
        }
    }
}

// Shadow rays: from the hit point toward the point light, restarted into
// the side of the hit triangle that faces the light, tmax = the distance.
__global__ void __launch_bounds__(kScanBlock)
emit_shadow_kernel(const __grid_constant__ MeshView mv, const tm_hit *__restrict__ hits, int64_t n,
                   const int64_t *n_dev, const int64_t *__restrict__ offsets, float lx, float ly,
                   float lz, tm_ray *__restrict__ out, int32_t *__restrict__ src) {
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    const HitIn h = load_hit(hits, i, valid_count(n, n_dev), mv.nc);
    const int64_t pos = hit_position(h.hit, offsets);
    if (!h.hit) return;
    const int32_t c = h.h1.y;
    const HitGeom g = hit_geometry(mv, h);
    const float facing = g.nx * (lx - g.a.x) + g.ny * (ly - g.a.y) + g.nz * (lz - g.a.z);
    const int side = facing >= 0.f ? 0 : 1;
    float vx = lx - g.ox, vy = ly - g.oy, vz = lz - g.oz;
    const float len = sqrtf(vx * vx + vy * vy + vz * vz);
    if (len > 0.f) {
        const float il = 1.f / len;
        vx *= il; vy *= il; vz *= il;
    } else {  // the light sits on the hit point: an empty segment along the normal
        const float il = (side ? -1.f : 1.f) / sqrtf(g.nx * g.nx + g.ny * g.ny + g.nz * g.nz);
        vx = g.nx * il; vy = g.ny * il; vz = g.nz * il;
    }
    put_ray(out, pos, g.ox, g.oy, g.oz, -1 - (2 * c + side), vx, vy, vz, len);
    if (src) src[pos] = (int32_t)i;
}

// Reflection / refraction rays (directions in the header's notation).
__global__ void __launch_bounds__(kScanBlock)
emit_specular_kernel(const __grid_constant__ MeshView mv, const tm_ray *__restrict__ rays_in,
                     const tm_hit *__restrict__ hits, int64_t n, const int64_t *n_dev,
                     const int64_t *__restrict__ offsets, int kind, float ior, float tmax,
                     tm_ray *__restrict__ out, int32_t *__restrict__ src) {
    const int64_t i = blockIdx.x * (int64_t)kScanBlock + threadIdx.x;
    const HitIn h = load_hit(hits, i, valid_count(n, n_dev), mv.nc);
    const int64_t pos = hit_position(h.hit, offsets);
    if (!h.hit) return;
    const int32_t c = h.h1.y;
    const int side = (h.h1.w & TM_HIT_SIDE_NEG) ? 1 : 0;  // arrival side
    const HitGeom g = hit_geometry(mv, h);
    const float4 din = __ldg(reinterpret_cast<const float4 *>(rays_in + i) + 1);
    const float iw = 1.f / sqrtf(din.x * din.x + din.y * din.y + din.z * din.z);
    const float wx = din.x * iw, wy = din.y * iw, wz = din.z * iw;
    const float in = (side ? -1.f : 1.f) / sqrtf(g.nx * g.nx + g.ny * g.ny + g.nz * g.nz);
    const float nx = g.nx * in, ny = g.ny * in, nz = g.nz * in;  // toward the arrival side
    const float cs = fmaxf(0.f, -(wx * nx + wy * ny + wz * nz));
    float dx, dy, dz;
    int out_side = side;
    const float eta = side ? ior : 1.f / ior;
    const float k = 1.f - eta * eta * (1.f - cs * cs);
    if (kind == TM_SPECULAR_REFRACT && k >= 0.f) {
        const float f = eta * cs - sqrtf(k);
        dx = eta * wx + f * nx;
        dy = eta * wy + f * ny;
        dz = eta * wz + f * nz;
        out_side = 1 - side;
    } else {
        dx = wx + 2.f * cs * nx;
        dy = wy + 2.f * cs * ny;
        dz = wz + 2.f * cs * nz;
    }
    const float il = 1.f / sqrtf(dx * dx + dy * dy + dz * dz);
    put_ray(out, pos, g.ox, g.oy, g.oz, -1 - (2 * c + out_side), dx * il, dy * il, dz * il, tmax);
    if (src) src[pos] = (int32_t)i;
}

}  // namespace tmk

tm_status launch_gen_primary(const tm_camera *cam, const int32_t *start, float tmax, tm_ray *rays,
                             cudaStream_t s) {
    const int64_t n = (int64_t)cam->width * cam->height;
    if (n == 0) return TM_OK;
    const int64_t tiles_x = ((int64_t)cam->width + tmk::kTileW - 1) / tmk::kTileW;
    const int64_t tiles_y = ((int64_t)cam->height + tmk::kTileH - 1) / tmk::kTileH;
    const int64_t gx = (tiles_x + 7) / 8;                    // eight tiles (warps) a block
    if (gx > INT32_MAX) return TM_ERR_TOO_LARGE;
    const dim3 grid((unsigned)gx, (unsigned)(tiles_y < 65535 ? tiles_y : 65535));
    tmk::gen_primary_kernel<<<grid, 256, 0, s>>>(*cam, start, tmax, rays);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        tm_set_error("gen_primary_kernel launch", e);
        return TM_ERR_CUDA;
    }
    tm_count_launches(1);
    return TM_OK;
}

namespace {

// Count, scan and emit with cudaMallocAsync scratch: `buckets` counts per
// block (one, or kLengthBuckets for the diffuse / occlusion generator);
// `count_pass(nb, counts)` launches the count kernel when given, else the
// plain hit count; `emit(nb, offsets)` launches the emit kernel.
template <class Emit, class Count>
tm_status gen_from_hits(const tm_hit *hits, int64_t n, const int64_t *n_dev, int32_t nc, int per_hit,
                        int64_t *count, cudaStream_t s, const char *what, Emit emit, int buckets,
                        Count count_pass) {
    using tmk::kScanBlock;
    if (n == 0) {
        TM_CUDA(cudaMemsetAsync(count, 0, sizeof(int64_t), s));
        return TM_OK;
    }
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb > INT32_MAX / tmk::kLengthBuckets) return TM_ERR_TOO_LARGE;
    int32_t *counts = nullptr;
    int64_t *offsets = nullptr;
    TM_CUDA(cudaMallocAsync((void **)&counts, sizeof(int32_t) * nb * buckets, s));
    cudaError_t ea = cudaMallocAsync((void **)&offsets, sizeof(int64_t) * (nb * buckets + 1), s);
    if (ea != cudaSuccess) {
        cudaFreeAsync(counts, s);
        tm_set_error("cudaMallocAsync (scan offsets)", ea);
        return TM_ERR_CUDA;
    }
    if (buckets > 1)
        count_pass((int)nb, counts);
    else
        tmk::count_hits_kernel<<<(int)nb, kScanBlock, 0, s>>>(hits, n, n_dev, nc, counts);
    tmk::scan_counts_kernel<<<1, kScanBlock, 0, s>>>(counts, nb * buckets, offsets, per_hit, count);
    emit((int)nb, offsets);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(counts, s);
    cudaFreeAsync(offsets, s);
    if (e != cudaSuccess) {
        tm_set_error(what, e);
        return TM_ERR_CUDA;
    }
    tm_count_launches(3);
    return TM_OK;
}

}  // namespace

tm_status launch_gen_shadow(const MeshView &mv, const tm_hit *hits, int64_t n, const int64_t *n_dev,
                            float lx, float ly, float lz, tm_ray *out, int64_t *count, int32_t *src,
                            cudaStream_t s) {
    return gen_from_hits(hits, n, n_dev, mv.nc, 1, count, s, "gen_shadow launch",
                         [&](int nb, const int64_t *offsets) {
                             tmk::emit_shadow_kernel<<<nb, tmk::kScanBlock, 0, s>>>(
                                 mv, hits, n, n_dev, offsets, lx, ly, lz, out, src);
                         }, 1, [](int, int32_t *) {});
}

tm_status launch_gen_specular(const MeshView &mv, const tm_ray *rays_in, const tm_hit *hits,
                              int64_t n, const int64_t *n_dev, int kind, float ior, float tmax,
                              tm_ray *out, int64_t *count, int32_t *src, cudaStream_t s) {
    return gen_from_hits(hits, n, n_dev, mv.nc, 1, count, s, "gen_specular launch",
                         [&](int nb, const int64_t *offsets) {
                             tmk::emit_specular_kernel<<<nb, tmk::kScanBlock, 0, s>>>(
                                 mv, rays_in, hits, n, n_dev, offsets, kind, ior, tmax, out, src);
                         }, 1, [](int, int32_t *) {});
}

tm_status launch_gen_secondary(const MeshView &mv, const tm_hit *hits, int64_t n,
                               const int64_t *n_dev, int per_hit, float tmax, uint64_t seed,
                               tm_ray *out, int64_t *count, int32_t *src, cudaStream_t s) {
    return gen_from_hits(hits, n, n_dev, mv.nc, per_hit, count, s, "gen_secondary launch",
                         [&](int nb, const int64_t *offsets) {
                             tmk::emit_secondary_kernel<<<nb, tmk::kEmitThreads, 0, s>>>(
                                 mv, hits, n, n_dev, offsets, per_hit, tmax, seed, out, src);
                         }, tmk::kLengthBuckets, [&](int nb, int32_t *counts) {
                             tmk::count_secondary_kernel<<<nb, tmk::kCountThreads, 0, s>>>(
                                 mv, hits, n, n_dev, per_hit, tmax, seed, counts);
                         });
}

// ---------------------------------------------------------------------------
// Secondary-ray generation without allocation.
//
// Some callers cannot allocate device memory while they run, e.g. a renderer
// that owns a fixed memory budget or code running inside a stream capture
// that must not create allocation nodes.  tm_gen_secondary_noalloc does the
// same work as tm_gen_secondary, but its scan scratch (per-block hit counts
// and offsets) lives in the static device array below instead of
// cudaMallocAsync memory.  The array holds the scratch for at most
// TM_NOALLOC_MAX_HITS hits, about 1.5 MiB, and stays on every device that
// loads this library until the process exits.
//
// The array is shared by every call: calls whose work overlaps on the GPU
// (other streams, other host threads) race on it.  Nothing in it needs to
// start at zero; each call writes every entry it later reads.
namespace {

constexpr int64_t kNoallocBlocks = (TM_NOALLOC_MAX_HITS + tmk::kScanBlock - 1) / tmk::kScanBlock;
constexpr int64_t kNoallocCounts = kNoallocBlocks * tmk::kLengthBuckets;
constexpr size_t kNoallocCountBytes = ((sizeof(int32_t) * kNoallocCounts + 255) / 256) * 256;
constexpr size_t kNoallocBytes = kNoallocCountBytes + sizeof(int64_t) * (kNoallocCounts + 1);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the host-side symbol is only a stand-in and is never passed to
// a kernel).
tm_status noalloc_scratch(void **addr) {
    int dev = 0;
    TM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        tm_set_error_text("tm_gen_secondary_noalloc: device ordinal out of range");
        return TM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) {
            tm_set_error("cudaGetSymbolAddress(g_noalloc_scratch)", e);
            return TM_ERR_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *addr = g_noalloc_addr[dev];
    return TM_OK;
}

}  // namespace

tm_status launch_gen_secondary_noalloc(const MeshView &mv, const tm_hit *hits, int64_t n,
                                       const int64_t *n_dev, int per_hit, float tmax, uint64_t seed,
                                       tm_ray *out, int64_t *count, int32_t *src, cudaStream_t s) {
    using tmk::kScanBlock;
    if (n > TM_NOALLOC_MAX_HITS) {
        tm_set_error_text("tm_gen_secondary_noalloc: " + std::to_string(n) +
                          " hits exceed the static scratch capacity of " +
                          std::to_string((long long)TM_NOALLOC_MAX_HITS));
        return TM_ERR_TOO_LARGE;
    }
    void *base = nullptr;
    const tm_status st = noalloc_scratch(&base);
    if (st != TM_OK) return st;
    if (n == 0) {
        TM_CUDA(cudaMemsetAsync(count, 0, sizeof(int64_t), s));
        return TM_OK;
    }
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    int32_t *counts = static_cast<int32_t *>(base);
    int64_t *offsets = reinterpret_cast<int64_t *>(static_cast<unsigned char *>(base) + kNoallocCountBytes);
    tmk::count_secondary_kernel<<<(int)nb, tmk::kCountThreads, 0, s>>>(mv, hits, n, n_dev, per_hit, tmax, seed,
                                                               counts);
    tmk::scan_counts_kernel<<<1, kScanBlock, 0, s>>>(counts, nb * tmk::kLengthBuckets, offsets, per_hit,
                                                     count);
    tmk::emit_secondary_kernel<<<(int)nb, tmk::kEmitThreads, 0, s>>>(mv, hits, n, n_dev, offsets, per_hit,
                                                             tmax, seed, out, src);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        tm_set_error("gen_secondary (no allocation) launch", e);
        return TM_ERR_CUDA;
    }
    tm_count_launches(3);
    return TM_OK;
}
