// Device arithmetic of the 2-D exit-face walk (Sec. 4 of the paper).
//
//  * Basis (Sec. 4.1, Eq. 1-2): for ray direction d with smallest |d| at
//    index mn and largest at mx, u_mn = 0, u_{mn+1} = d_{mn+2}/d_mx,
//    u_{mn+2} = -d_{mn+1}/d_mx (indices mod 3, non-negative), so the
//    component of u at the remaining index is exactly +-1; t = d x u and
//    v = t / |t_mn|, so v_mn = +-1 exactly (the "+-" of Eq. 3) and
//    (u, v, d) is right-handed.  Scaling the basis leaves every exit
//    decision unchanged (Sec. 4.1).
//  * Projected origin (Sec. 7, optimisation 1): po = (u.o, v.o); a point x
//    projects to p = (u.x - po_x, v.x - po_y), with the same fused
//    multiply-add chain for po and for every point, so the origin itself
//    projects to (0, 0) exactly.
//  * Sign tests: det(a, b) = a.x*b.y - a.y*b.x with separately rounded
//    products, hence det(b, a) = -det(a, b) bit for bit; an exact zero is
//    broken by vertex ids (the pair decides as if id_a < id_b gave +), so a
//    pair of vertices gets the same answer in every tet of a ray's walk.
//    In guard mode a test with |det| < tau * max|coordinate| is re-decided
//    in double precision from the 3-D points: with A = a - o and B = b - o,
//    det(P(a), P(b)) = (u.A)(v.B) - (v.A)(u.B) = (A x B).(u x v) (Binet-
//    Cauchy), and u x v = (|u|^2 / |t_min|) d points along d, so the sign is
//    that of the triple product (A x B).d: no basis, no division.
//  * Exit face (Alg. 1): with the entry face p0, p1, p2 counter-clockwise
//    around the origin, the new vertex p3 replaces slot e, and the kept
//    face is again counter-clockwise (Sec. 4: replacing a slot keeps the
//    winding, so no reordering is ever needed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tm_internal.h"

namespace tmk {

enum : int { FP32G = TM_MODE_FP32_GUARD, FP32 = TM_MODE_FP32, FP64 = TM_MODE_FP64 };

// Vertex slot j of local face k (opposite V_k) of a positively oriented
// tet, ordered so that the face normal points into the tet:
// {1,3,2}, {0,2,3}, {0,3,1}, {0,1,2}.  A function so that unrolled loops
// fold it to constants.
__host__ __device__ __forceinline__ constexpr int face_in(int k, int j) {
    return k == 0 ? (j == 0 ? 1 : (j == 1 ? 3 : 2))
         : k == 1 ? (j == 0 ? 0 : (j == 1 ? 2 : 3))
         : k == 2 ? (j == 0 ? 0 : (j == 1 ? 3 : 1))
                  : (j == 0 ? 0 : (j == 1 ? 1 : 2));
}

template <int MODE> struct RealOf { typedef float T; };
template <> struct RealOf<FP64> { typedef double T; };

template <class R> struct P2 { R x, y; };

__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class R> __device__ __forceinline__ R det2(const P2<R> &a, const P2<R> &b) {
    return rsub(rmul(a.x, b.y), rmul(a.y, b.x));
}

// det2 for float with both products in one packed two-wide multiply
// (mul.rn.f32x2, sm_100 and later): (a.y * b.x, a.x * b.y), then the
// difference of the halves.  Each product and the difference are rounded
// as in det2, so the result is the same bit for bit.
#ifndef TM_PACKED_DET
#define TM_PACKED_DET 1
#endif
__device__ __forceinline__ float det2_packed(const P2<float> &a, const P2<float> &b) {
#if TM_PACKED_DET
    unsigned long long A, B, Q;
    asm("mov.b64 %0, {%1, %2};" : "=l"(A) : "f"(a.y), "f"(a.x));
    asm("mov.b64 %0, {%1, %2};" : "=l"(B) : "f"(b.x), "f"(b.y));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(Q) : "l"(A), "l"(B));
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(Q));
    return __fsub_rn(hi, lo);
#else
    return det2(a, b);
#endif
}

template <class R> struct Basis {
    R ux, uy, uz, vx, vy, vz, pox, poy;

    __device__ __forceinline__ P2<R> project(R x, R y, R z) const {
        P2<R> p;
        p.x = rsub(rfma(uz, z, rfma(uy, y, rmul(ux, x))), pox);
        p.y = rsub(rfma(vz, z, rfma(vy, y, rmul(vx, x))), poy);
        return p;
    }
};

// Modified basis of Eq. 1-2 for direction d, and the projected origin.
template <class R>
__device__ __forceinline__ Basis<R> make_basis(R dx, R dy, R dz, R ox, R oy, R oz) {
    const R ax = fabs(dx), ay = fabs(dy), az = fabs(dz);
    int mn = 0;
    if (ay < ax) mn = 1;
    if (az < (mn == 0 ? ax : ay)) mn = 2;
    int mx = 2;
    if (ay > az) mx = 1;
    if (ax > (mx == 2 ? az : ay)) mx = 0;
    // rotate so that the smallest component comes first: r = (d_mn, d_mn+1, d_mn+2)
    const R r0 = mn == 0 ? dx : (mn == 1 ? dy : dz);
    const R r1 = mn == 0 ? dy : (mn == 1 ? dz : dx);
    const R r2 = mn == 0 ? dz : (mn == 1 ? dx : dy);
    const R dmx = mx == 0 ? dx : (mx == 1 ? dy : dz);
    const R u1 = rdiv(r2, dmx), u2 = -rdiv(r1, dmx);          // u0 = 0
    const R t0 = rsub(rmul(r1, u2), rmul(r2, u1));            // t = r x u
    const R t1 = -rmul(r0, u2);
    const R t2 = rmul(r0, u1);
    const R at0 = fabs(t0);
    const R v0 = t0 < R(0) ? R(-1) : R(1);
    const R v1 = rdiv(t1, at0), v2 = rdiv(t2, at0);
    Basis<R> b;
    // rotate back: component mn + i (mod 3) takes rotated component i
    b.ux = mn == 0 ? R(0) : (mn == 1 ? u2 : u1);
    b.uy = mn == 0 ? u1 : (mn == 1 ? R(0) : u2);
    b.uz = mn == 0 ? u2 : (mn == 1 ? u1 : R(0));
    b.vx = mn == 0 ? v0 : (mn == 1 ? v2 : v1);
    b.vy = mn == 0 ? v1 : (mn == 1 ? v0 : v2);
    b.vz = mn == 0 ? v2 : (mn == 1 ? v1 : v0);
    b.pox = R(0);
    b.poy = R(0);
    const P2<R> po = b.project(ox, oy, oz);
    b.pox = po.x;
    b.poy = po.y;
    return b;
}

// ((a - o) x (b - o)) . d in double precision from the float32 inputs: a
// positive multiple of det(P(a), P(b)) in the ray's basis (see the header).
__device__ __forceinline__ double triple(const float4 &o, const float4 &d, const float4 &a,
                                         const float4 &b) {
    const double ax = (double)a.x - o.x, ay = (double)a.y - o.y, az = (double)a.z - o.z;
    const double bx = (double)b.x - o.x, by = (double)b.y - o.y, bz = (double)b.z - o.z;
    const double cx = ay * bz - az * by, cy = az * bx - ax * bz, cz = ax * by - ay * bx;
    return cx * d.x + cy * d.y + cz * d.z;
}

// Double-precision sign decision of det(p_a, p_b) for two float32 points of
// one ray (the guard's re-test).  Out of line by default: it is the rare path.
#ifdef TM_GUARD_INLINE
#define TM_GUARD_ATTR __forceinline__
#else
#define TM_GUARD_ATTR __noinline__
#endif
__device__ TM_GUARD_ATTR static double guard_det(const tm_ray *ray, const float4 *pts, int32_t ia,
                                                int32_t ib) {
    const float4 w0 = __ldg(reinterpret_cast<const float4 *>(ray));
    const float4 w1 = __ldg(reinterpret_cast<const float4 *>(ray) + 1);
    return triple(w0, w1, __ldg(pts + ia), __ldg(pts + ib));
}

// tau * max(|p.x|, |p.y|): the guard threshold contribution of one point.
template <class R> __device__ __forceinline__ float guard_mag(const P2<R> &p, float tau) {
    return tau * fmaxf(fabsf((float)p.x), fabsf((float)p.y));
}

// Everything the sign tests of one ray need besides the two points.
struct SignCtx {
    const tm_ray *ray;
    const float4 *pts;
    float tau;       // guard threshold in scene units (guard_tau * extent)
    uint32_t flags;  // TM_HIT_GUARD / TM_HIT_TIE accumulate here
};

// Consistent orientation: true when (origin, a, b) turns counter-clockwise,
// i.e. det(a, b) > 0, with ties broken by the vertex ids.
template <int MODE, class R>
__device__ __forceinline__ bool pos(const P2<R> &a, const P2<R> &b, int32_t ia, int32_t ib,
                                    SignCtx &c) {
    const R d = det2(a, b);
    if (MODE == FP32G) {
        // threshold tau * max|coordinate| of the pair, the same rule as step_signs()
        const float t = fmaxf(guard_mag(a, c.tau), guard_mag(b, c.tau));
        if (!(fabsf((float)d) > t)) {
            c.flags |= TM_HIT_GUARD;
            const double dd = guard_det(c.ray, c.pts, ia, ib);
            if (dd != 0.0) return dd > 0.0;
            c.flags |= TM_HIT_TIE;
            return ia < ib;
        }
        return d > R(0);
    }
    if (d != R(0)) return d > R(0);
    c.flags |= TM_HIT_TIE;
    return ia < ib;
}

// Alg. 1: slot (0, 1, 2) of the entry face that the new vertex replaces.
template <int MODE, class R>
__device__ __forceinline__ int exit_slot(const P2<R> &p0, const P2<R> &p1, const P2<R> &p2,
                                         const P2<R> &p3, int32_t i0, int32_t i1, int32_t i2,
                                         int32_t i3, SignCtx &c) {
    if (!pos<MODE>(p3, p0, i3, i0, c)) return pos<MODE>(p3, p2, i3, i2, c) ? 1 : 0;
    return pos<MODE>(p3, p1, i3, i1, c) ? 0 : 2;
}

// Walk state of one ray: the current tet, the tet it came from, and the
// face it entered through (ids and projections, counter-clockwise).
template <class R> struct WalkState {
    int32_t tet, prev;
    int32_t i0, i1, i2;
    P2<R> p0, p1, p2;
    float m0, m1, m2;  // guard mode: tau * max(|p.x|, |p.y|) of each slot
    // face-entry walk: the current tet's fourth vertex, known on entering it
    int32_t i3;
    P2<R> p3;
    float m3;
};



// Exit face of tet T for the ray's line (Sec. 4: the first tet needs up to
// four 2-D triangle tests): the face, other than `skip`, whose projection
// holds the origin with clockwise order in its inward orientation.  On
// success fills the state (entry face of the next tet, counter-clockwise)
// and returns the raw neighbour value across it; returns false when no
// face or more than one face qualifies.
template <int MODE, class R>
__device__ __forceinline__ bool line_init_core(const Basis<R> &B, int32_t T, int skip,
                                               const int32_t (&V)[4], const uint32_t (&NB)[4],
                                               const float (&X)[4][3], SignCtx &c, WalkState<R> &S,
                                               uint32_t &next) {
    P2<R> P[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) P[k] = B.project(X[k][0], X[k][1], X[k][2]);
    // The six edges' orientations, each decided once; a face that runs an
    // edge the other way reads the negation, so the four faces agree on
    // every edge whatever the rounding of the re-test.
    bool s[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = i + 1; j < 4; ++j) s[i][j] = pos<MODE>(P[i], P[j], V[i], V[j], c);
    auto ccw = [&](int i, int j) { return i < j ? s[i][j] : !s[j][i]; };
    int found = -1, count = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k == skip) continue;
        const int a = face_in(k, 0), b = face_in(k, 1), d = face_in(k, 2);
        const bool cw = !ccw(a, b) && !ccw(b, d) && !ccw(d, a);
        if (cw) {
            if (found < 0) found = k;
            ++count;
        }
    }
    if (count != 1) return false;
    // counter-clockwise order of the exit face: reverse its inward order
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k == found) {
            const int a = face_in(k, 0), b = face_in(k, 1), d = face_in(k, 2);
            S.i0 = V[a]; S.p0 = P[a];
            S.i1 = V[d]; S.p1 = P[d];
            S.i2 = V[b]; S.p2 = P[b];
            next = NB[k];
        }
    }
    S.prev = T;
    S.m0 = guard_mag(S.p0, c.tau);
    S.m1 = guard_mag(S.p1, c.tau);
    S.m2 = guard_mag(S.p2, c.tau);
    return true;
}

// line_init_core on tet T read from its cold record and the points.
template <int MODE, class R>
__device__ __forceinline__ bool line_init(const MeshView &mv, const Basis<R> &B, int32_t T, int skip,
                                          SignCtx &c, WalkState<R> &S, uint32_t &next) {
    const int4 cv = __ldg(mv.cold + 2 * T);
    const int4 cn = __ldg(mv.cold + 2 * T + 1);
    const int32_t V[4] = {cv.x, cv.y, cv.z, cv.w};
    const uint32_t NB[4] = {(uint32_t)cn.x, (uint32_t)cn.y, (uint32_t)cn.z, (uint32_t)cn.w};
    float X[4][3];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 x = __ldg(mv.pts + V[k]);
        X[k][0] = x.x; X[k][1] = x.y; X[k][2] = x.z;
    }
    return line_init_core<MODE>(B, T, skip, V, NB, X, c, S, next);
}

// line_init_core on the restart record of triangle side (2c + side): the
// tet on that side with its ids, neighbours and vertex positions inline, so
// a restarted ray reaches its line test after one read.  Six int4:
// {V0..V3}, {N0..N3}, {x0 y0 z0 x1}, {y1 z1 x2 y2}, {z2 x3 y3 z3}, {T, skip, 0, 0}.
// Returns false with T = -1 when the side has no tet.
template <int MODE, class R>
__device__ __forceinline__ bool restart_init(const MeshView &mv, const Basis<R> &B, int64_t rec,
                                             int32_t &T, int &skip, SignCtx &c, WalkState<R> &S,
                                             uint32_t &next) {
    const int4 *r = mv.restart + 6 * rec;
    const int4 cv = __ldg(r), cn = __ldg(r + 1), g0 = __ldg(r + 2), g1 = __ldg(r + 3),
               g2 = __ldg(r + 4), h = __ldg(r + 5);
    T = h.x;
    skip = h.y;
    if (T < 0 || T >= mv.nt || skip < 0 || skip > 3) {
        T = -1;
        return false;
    }
    const int32_t V[4] = {cv.x, cv.y, cv.z, cv.w};
    const uint32_t NB[4] = {(uint32_t)cn.x, (uint32_t)cn.y, (uint32_t)cn.z, (uint32_t)cn.w};
    const float X[4][3] = {{__int_as_float(g0.x), __int_as_float(g0.y), __int_as_float(g0.z)},
                           {__int_as_float(g0.w), __int_as_float(g1.x), __int_as_float(g1.y)},
                           {__int_as_float(g1.z), __int_as_float(g1.w), __int_as_float(g2.x)},
                           {__int_as_float(g2.y), __int_as_float(g2.z), __int_as_float(g2.w)}};
    return line_init_core<MODE>(B, T, skip, V, NB, X, c, S, next);
}

// The rare restart fallback: one 3-D face-plane step in double precision
// (exit through the face plane with the smallest positive crossing, the
// entry face excluded), used only when the line misses the restart tet by
// rounding.  Returns the raw neighbour value crossed (x) and the local index
// of the shared face inside the neighbour (y, or -1).
__device__ __noinline__ static int2 step3d(const MeshView &mv, const tm_ray *ray, int32_t T,
                                           int skip) {
    const float4 w0 = __ldg(reinterpret_cast<const float4 *>(ray));
    const float4 w1 = __ldg(reinterpret_cast<const float4 *>(ray) + 1);
    const double o[3] = {w0.x, w0.y, w0.z}, d[3] = {w1.x, w1.y, w1.z};
    const int4 cv = __ldg(mv.cold + 2 * T), cn = __ldg(mv.cold + 2 * T + 1);
    const int32_t V[4] = {cv.x, cv.y, cv.z, cv.w};
    const uint32_t NB[4] = {(uint32_t)cn.x, (uint32_t)cn.y, (uint32_t)cn.z, (uint32_t)cn.w};
    double X[4][3];
    for (int k = 0; k < 4; ++k) {
        const float4 x = __ldg(mv.pts + V[k]);
        X[k][0] = x.x; X[k][1] = x.y; X[k][2] = x.z;
    }
    int best = -1;
    double tb = 0.0;
    for (int k = 0; k < 4; ++k) {
        if (k == skip) continue;
        const double *a = X[face_in(k, 0)], *b = X[face_in(k, 1)], *e = X[face_in(k, 2)];
        const double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double ae[3] = {e[0] - a[0], e[1] - a[1], e[2] - a[2]};
        const double n[3] = {ab[1] * ae[2] - ab[2] * ae[1], ab[2] * ae[0] - ab[0] * ae[2],
                             ab[0] * ae[1] - ab[1] * ae[0]};
        const double nd = n[0] * d[0] + n[1] * d[1] + n[2] * d[2];
        if (nd < 0.0) {
            const double tk = (n[0] * (a[0] - o[0]) + n[1] * (a[1] - o[1]) + n[2] * (a[2] - o[2])) / nd;
            if (best < 0 || tk < tb) { best = k; tb = tk; }
        }
    }
    int skip_next = -1;
    if (best < 0) return make_int2((int)TM_BOUNDARY, -1);
    const uint32_t nb = NB[best];
    if (!(nb & TM_CFACE_FLAG) && nb < (uint32_t)mv.nt) {
        const int4 un = __ldg(mv.cold + 2 * (int32_t)nb + 1);
        const int32_t UN[4] = {un.x, un.y, un.z, un.w};
        for (int k = 0; k < 4; ++k)
            if (UN[k] == T) skip_next = k;
    }
    return make_int2((int)nb, skip_next);
}

// The sign tests of one step, det(p3, p_k) > 0 for the entry-face slots
// k = 0, 1, 2 (bit k), with the same decision rule as pos().  In guard mode
// only the two tests Alg. 1 reads are made (and guarded); with PARK a step
// with an ambiguous one is not decided: the function returns kParked and the
// caller hands the ray to the slow pass; INLINE_GUARD inlines the
// double-precision re-test instead of calling it.
constexpr uint32_t kParked = 0xffffffffu;

// Guard mode: the double-precision decision of one sign test det(p_a, p_b)
// (ties broken by ids), with TM_HIT_GUARD / TM_HIT_TIE added to *flags.
template <bool INLINE>
__device__ __forceinline__ bool guard_one(const tm_ray *ray, const float4 *pts, int32_t ia, int32_t ib,
                                          uint32_t &flags) {
    double dd;
    if (INLINE) {
        const float4 w0 = __ldg(reinterpret_cast<const float4 *>(ray));
        const float4 w1 = __ldg(reinterpret_cast<const float4 *>(ray) + 1);
        dd = triple(w0, w1, __ldg(pts + ia), __ldg(pts + ib));
    } else {
        dd = guard_det(ray, pts, ia, ib);
    }
    flags |= TM_HIT_GUARD;
    if (dd != 0.0) return dd > 0.0;
    flags |= TM_HIT_TIE;
    return ia < ib;
}

template <int MODE, bool PARK, bool INLINE_GUARD, class R>
__device__ __forceinline__ uint32_t step_signs(const WalkState<R> &S, const P2<R> &p3, int32_t i3,
                                               float m3, SignCtx &c) {
    if (MODE == FP32G) {
        // Alg. 1 reads two sign tests: det(p3, p0), then det(p3, p1) when it is
        // positive, det(p3, p2) otherwise; only those two are guarded.  The
        // bits returned give exit_slot_bits() the same slot.
        const R d0 = det2(p3, S.p0);
        bool s0 = d0 > R(0);
        if (!(fabsf((float)d0) > fmaxf(m3, S.m0))) {
            if (PARK) return kParked;
            s0 = guard_one<INLINE_GUARD>(c.ray, c.pts, i3, S.i0, c.flags);
        }
        const P2<R> pk = s0 ? S.p1 : S.p2;
        const R dk = det2(p3, pk);
        bool sk = dk > R(0);
        if (!(fabsf((float)dk) > fmaxf(m3, s0 ? S.m1 : S.m2))) {
            if (PARK) return kParked;
            sk = guard_one<INLINE_GUARD>(c.ray, c.pts, i3, s0 ? S.i1 : S.i2, c.flags);
        }
        return s0 ? (1u | ((uint32_t)sk << 1)) : ((uint32_t)sk << 2);
    }
    const R d0 = det2(p3, S.p0), d1 = det2(p3, S.p1), d2 = det2(p3, S.p2);
    uint32_t bits = (uint32_t)(d0 > R(0)) | ((uint32_t)(d1 > R(0)) << 1) | ((uint32_t)(d2 > R(0)) << 2);
    if ((d0 == R(0)) | (d1 == R(0)) | (d2 == R(0))) {
        c.flags |= TM_HIT_TIE;
        if (d0 == R(0)) bits |= (uint32_t)(i3 < S.i0);
        if (d1 == R(0)) bits |= (uint32_t)(i3 < S.i1) << 1;
        if (d2 == R(0)) bits |= (uint32_t)(i3 < S.i2) << 2;
    }
    return bits;
}

// Alg. 1 on the three signs: slot (0, 1, 2) that the new vertex replaces.
__device__ __forceinline__ int exit_slot_bits(uint32_t s) {
    return (s & 1u) ? ((s & 2u) ? 0 : 2) : ((s & 4u) ? 1 : 0);
}

// Does the closed tet T hold the ray origin (double precision, with a
// relative tolerance for points on its faces)?
__device__ __noinline__ static bool holds_origin(const MeshView &mv, const tm_ray *ray, int32_t T) {
    const float4 w0 = __ldg(reinterpret_cast<const float4 *>(ray));
    const double o[3] = {w0.x, w0.y, w0.z};
    const int4 cv = __ldg(mv.cold + 2 * T);
    const int32_t V[4] = {cv.x, cv.y, cv.z, cv.w};
    double X[4][3];
    for (int k = 0; k < 4; ++k) {
        const float4 x = __ldg(mv.pts + V[k]);
        X[k][0] = x.x; X[k][1] = x.y; X[k][2] = x.z;
    }
    for (int k = 0; k < 4; ++k) {
        const double *a = X[face_in(k, 0)], *b = X[face_in(k, 1)], *c = X[face_in(k, 2)];
        const double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double ac[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const double n[3] = {ab[1] * ac[2] - ab[2] * ac[1], ab[2] * ac[0] - ab[0] * ac[2],
                             ab[0] * ac[1] - ab[1] * ac[0]};
        const double side = n[0] * (o[0] - a[0]) + n[1] * (o[1] - a[1]) + n[2] * (o[2] - a[2]);
        const double scale = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (side < -1e-12 * scale) return false;  // strictly outside the plane of face k
    }
    return true;
}

// Final ray-triangle test on the hit triangle in its own vertex order
// (Moller & Trumbore 1997): t and (b1, b2).  `cond` estimates how many
// units of rounding the computed t may be off by (relative): the condition
// numbers of t's denominator d.(e2 x e1) and numerator s.(e1 x e2), measured
// with 1-norms, so cond * eps bounds the relative error of t up to a small
// constant.  It is large for grazing rays and for origins close to the
// triangle's plane far from its vertices.
template <class R>
__device__ __forceinline__ void mt_hit(const float4 &o4, const float4 &d4, const float4 &a4,
                                       const float4 &b4, const float4 &c4, R &t, R &b1, R &b2,
                                       R &cond) {
    const R e1x = R(b4.x) - R(a4.x), e1y = R(b4.y) - R(a4.y), e1z = R(b4.z) - R(a4.z);
    const R e2x = R(c4.x) - R(a4.x), e2y = R(c4.y) - R(a4.y), e2z = R(c4.z) - R(a4.z);
    const R dx = d4.x, dy = d4.y, dz = d4.z;
    const R px = dy * e2z - dz * e2y, py = dz * e2x - dx * e2z, pz = dx * e2y - dy * e2x;
    const R det = e1x * px + e1y * py + e1z * pz;
    const R sx = R(o4.x) - R(a4.x), sy = R(o4.y) - R(a4.y), sz = R(o4.z) - R(a4.z);
    const R qx = sy * e1z - sz * e1y, qy = sz * e1x - sx * e1z, qz = sx * e1y - sy * e1x;
    const R num = e2x * qx + e2y * qy + e2z * qz;
    const R inv = R(1) / det;
    b1 = (sx * px + sy * py + sz * pz) * inv;
    b2 = (dx * qx + dy * qy + dz * qz) * inv;
    t = num * inv;
    const R n1 = (fabs(e1x) + fabs(e1y) + fabs(e1z)) * (fabs(e2x) + fabs(e2y) + fabs(e2z));
    cond = n1 * ((fabs(dx) + fabs(dy) + fabs(dz)) / fabs(det) + (fabs(sx) + fabs(sy) + fabs(sz)) / fabs(num));
}

}  // namespace tmk
