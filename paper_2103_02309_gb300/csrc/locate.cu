// Point location (Sec. 4.2 of the paper: the traversal walk, used in 3-D,
// from a source tet).  For a query q, the walk follows the segment from the
// source tet's centroid c to q with the 2-D exit-face step of the ray
// traversal; constrained faces do not stop it (the flagged neighbour is
// crossed to the other tet of the face).  After each exit face is known, one
// 3-D orientation test decides whether q lies before that face's plane; if
// it does, q is in the current tet.  The walk runs in float32 first and, if
// it leaves the mesh or exceeds its bound, once more in double precision.
#include "walk.cuh"

namespace tmk {

// Sign of orient3d(a, b, c, q) (q on the side the normal (b-a)x(c-a) points
// to: > 0), float32 with a conservative error filter, else double.
__device__ __forceinline__ int orient_q(const float4 &a, const float4 &b, const float4 &c, float qx,
                                        float qy, float qz) {
    const float ax = a.x - qx, ay = a.y - qy, az = a.z - qz;
    const float bx = b.x - qx, by = b.y - qy, bz = b.z - qz;
    const float cx = c.x - qx, cy = c.y - qy, cz = c.z - qz;
    // det[a-q, b-q, c-q] = orient3d(q, a, b, c) = -orient3d(a, b, c, q)
    const float d = ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
    const float na = fabsf(ax) + fabsf(ay) + fabsf(az), nb = fabsf(bx) + fabsf(by) + fabsf(bz),
                nc = fabsf(cx) + fabsf(cy) + fabsf(cz);
    // rounding of the three differences (<= 2e-7 each in the 1-norm for
    // coordinates of magnitude <= 1) plus that of the products
    const float bound = 1e-6f * na * nb * nc + 4e-7f * (nb * nc + na * nc + na * nb);
    if (fabsf(d) > bound) return d > 0.f ? -1 : 1;
    const double Ax = (double)a.x - qx, Ay = (double)a.y - qy, Az = (double)a.z - qz;
    const double Bx = (double)b.x - qx, By = (double)b.y - qy, Bz = (double)b.z - qz;
    const double Cx = (double)c.x - qx, Cy = (double)c.y - qy, Cz = (double)c.z - qz;
    const double D = Ax * (By * Cz - Bz * Cy) + Ay * (Bz * Cx - Bx * Cz) + Az * (Bx * Cy - By * Cx);
    return D > 0.0 ? -1 : (D < 0.0 ? 1 : 0);
}

// q lies on the inner side of (or on) the exit face kept in S, whose
// counter-clockwise 2-D order (i0, i1, i2) is the outward order, so
// (i0, i2, i1) is the inward one.
__device__ __forceinline__ bool before_exit(const MeshView &mv, int32_t i0, int32_t i1, int32_t i2,
                                            float qx, float qy, float qz) {
    const float4 a = __ldg(mv.pts + i0), b = __ldg(mv.pts + i2), c = __ldg(mv.pts + i1);
    return orient_q(a, b, c, qx, qy, qz) >= 0;
}

// Returns the tet holding q, -1 when q is outside the mesh, -2 when the walk
// failed (bound exceeded or no exit face).
template <int MODE>
__device__ int32_t locate_walk(const MeshView &mv, int32_t T, float qx, float qy, float qz,
                               uint32_t max_steps) {
    typedef typename RealOf<MODE>::T R;
    const int4 cv = __ldg(mv.cold + 2 * T);
    const float4 x0 = __ldg(mv.pts + cv.x), x1 = __ldg(mv.pts + cv.y), x2 = __ldg(mv.pts + cv.z),
                 x3 = __ldg(mv.pts + cv.w);
    const float cx = ((x0.x + x1.x) + (x2.x + x3.x)) * 0.25f;
    const float cy = ((x0.y + x1.y) + (x2.y + x3.y)) * 0.25f;
    const float cz = ((x0.z + x1.z) + (x2.z + x3.z)) * 0.25f;
    const R dx = R(qx) - R(cx), dy = R(qy) - R(cy), dz = R(qz) - R(cz);
    if (dx == R(0) && dy == R(0) && dz == R(0)) return T;
    const Basis<R> B = make_basis<R>(dx, dy, dz, R(cx), R(cy), R(cz));
    SignCtx sc;
    sc.ray = nullptr;
    sc.pts = mv.pts;
    sc.tau = 0.f;
    sc.flags = 0;
    WalkState<R> S;
    uint32_t next;
    if (!line_init<MODE == FP64 ? FP64 : FP32>(mv, B, T, -1, sc, S, next)) return -2;
    for (uint32_t steps = 0;; ++steps) {
        // S.prev is the current tet, its exit face is (i0, i1, i2), `next` lies beyond it
        if (before_exit(mv, S.i0, S.i1, S.i2, qx, qy, qz)) return S.prev;
        if (steps >= max_steps) return -2;
        const int32_t cur = S.prev;
        int32_t nt;
        uint32_t prev_code;
        if (next & TM_CFACE_FLAG) {
            if (next == TM_BOUNDARY) return -1;
            const int32_t c = (int32_t)(next & ~TM_CFACE_FLAG);
            if (c >= mv.nc) return -2;
            const int4 r0 = __ldg(mv.cface + 2 * c);
            nt = (r0.y == cur) ? r0.z : r0.y;
            if (nt < 0) return -1;
            if (nt >= mv.nt) return -2;
            prev_code = next;  // the tet on the other side stores the same flagged value
        } else {
            if (next >= (uint32_t)mv.nt) return -2;
            nt = (int32_t)next;
            prev_code = (uint32_t)cur;
        }
        // one step of Alg. 6 / Alg. 7 in tet nt
        const int4 rec = __ldg(mv.tet16 + nt);
        const int32_t i3 = S.i0 ^ S.i1 ^ S.i2 ^ rec.x;
        if ((uint32_t)i3 >= (uint32_t)mv.np) return -2;
        const float4 x = __ldg(mv.pts + i3);
        const P2<R> p3 = B.project(R(x.x), R(x.y), R(x.z));
        const int e = exit_slot<MODE == FP64 ? FP64 : FP32>(S.p0, S.p1, S.p2, p3, S.i0, S.i1, S.i2, i3, sc);
        const int ra = (S.i0 < i3) + (S.i1 < i3) + (S.i2 < i3);
        const int32_t ie = e == 0 ? S.i0 : (e == 1 ? S.i1 : S.i2);
        const int rb = (S.i0 < ie) + (S.i1 < ie) + (S.i2 < ie) + (i3 < ie);
        const uint32_t nxa = ra == 0 ? rec.y : (ra == 1 ? rec.z : (ra == 2 ? rec.w : 0));
        const uint32_t nxb = rb == 0 ? rec.y : (rb == 1 ? rec.z : (rb == 2 ? rec.w : 0));
        next = prev_code ^ nxa ^ nxb;
        if (e == 0) { S.i0 = i3; S.p0 = p3; }
        else if (e == 1) { S.i1 = i3; S.p1 = p3; }
        else { S.i2 = i3; S.p2 = p3; }
        S.prev = nt;
    }
}

__global__ void __launch_bounds__(256)
locate_kernel(const __grid_constant__ MeshView mv, const float *__restrict__ q, int64_t n,
              const int32_t *__restrict__ hint, int32_t source, int32_t *__restrict__ out,
              uint32_t max_steps) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float qx = q[3 * i], qy = q[3 * i + 1], qz = q[3 * i + 2];
        int32_t T = hint ? hint[i] : -1;
        if ((T < 0 || T >= mv.nt) && mv.seeds) {
            // the located tet of the lattice cell that holds q
            const int G = kSeedGrid;
            const int ci = min(max((int)((qx - mv.lo[0]) * mv.cell_inv), 0), G - 1);
            const int cj = min(max((int)((qy - mv.lo[1]) * mv.cell_inv), 0), G - 1);
            const int ck = min(max((int)((qz - mv.lo[2]) * mv.cell_inv), 0), G - 1);
            T = __ldg(mv.seeds + ci + G * (cj + G * ck));
        }
        if (T < 0 || T >= mv.nt) T = source;
        int32_t r = locate_walk<FP32>(mv, T, qx, qy, qz, max_steps);
        if (r < 0) r = locate_walk<FP64>(mv, T, qx, qy, qz, max_steps);
        out[i] = r < 0 ? -1 : r;
    }
}

}  // namespace tmk

tm_status launch_locate(const MeshView &mv, const float *q, int64_t n, const int32_t *hint,
                        int32_t source, int32_t *out, uint32_t max_steps, cudaStream_t s) {
    if (n == 0) return TM_OK;
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = (n + 255) / 256;
    if (grid > (int64_t)sms * 8) grid = (int64_t)sms * 8;
    tmk::locate_kernel<<<(int)grid, 256, 0, s>>>(mv, q, n, hint, source, out, max_steps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        tm_set_error("locate_kernel launch", e);
        return TM_ERR_CUDA;
    }
    tm_count_launches(1);
    return TM_OK;
}
