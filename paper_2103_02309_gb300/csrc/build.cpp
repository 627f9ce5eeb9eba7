// Host construction of the compact mesh records (Sec. 3) and their Hilbert
// order (Sec. 5), then the upload to the device.
//
// Steps (tm_build):
//  1. validate ids and orientation (orient3d > 0 in double precision);
//  2. neighbours: every face keyed by its sorted vertex triple, bucketed by
//     the smallest vertex id, matched within its bucket;
//  3. constrained faces: each input triangle matched to its one or two tet
//     faces, whose neighbour fields are replaced by the flagged triangle id;
//     the tet whose opposite vertex lies on the + side of the triangle's own
//     plane becomes tet+, the other tet-;
//  4. Hilbert keys (3 x 21 bits) of point positions and tet centroids, a
//     stable sort, and the renumbering of every id; with regions (Sec. 5),
//     the tets are first grouped by the connected component of the
//     non-constrained face graph that holds them (a concurrent union-find);
//  5. packing: cold records (V0..V3, N0..N3) and Tet16 records
//     (VX = V0^V1^V2^V3; NX_j = N_j ^ N_3 with the neighbours sorted by the
//     id of the vertex they sit across, Sec. 3, the Tet20 and Tet16 layouts).
#include <omp.h>
#include <parallel/algorithm>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>

#include "tm_internal.h"

namespace {

double orient3d(const double *a, const double *b, const double *c, const double *d) {
    const double abx = b[0] - a[0], aby = b[1] - a[1], abz = b[2] - a[2];
    const double acx = c[0] - a[0], acy = c[1] - a[1], acz = c[2] - a[2];
    const double adx = d[0] - a[0], ady = d[1] - a[1], adz = d[2] - a[2];
    return (aby * acz - abz * acy) * adx + (abz * acx - abx * acz) * ady +
           (abx * acy - aby * acx) * adz;
}

// Local face k (opposite V_k) of a positively oriented tet, vertex slots
// ordered so that the face normal points into the tet.
const int kFaceIn[4][3] = {{1, 3, 2}, {0, 2, 3}, {0, 3, 1}, {0, 1, 2}};

struct FaceEntry {
    int32_t b, c;   // the two larger vertex ids of the face
    int32_t owner;  // 4*tet + k
};

inline void sort3(int32_t &x, int32_t &y, int32_t &z) {
    if (x > y) std::swap(x, y);
    if (y > z) std::swap(y, z);
    if (x > y) std::swap(x, y);
}

inline bool face_less(const FaceEntry &l, const FaceEntry &r) {
    if (l.b != r.b) return l.b < r.b;
    if (l.c != r.c) return l.c < r.c;
    return l.owner < r.owner;
}

}  // namespace

// 3-D Hilbert index of integer coordinates (bits per axis <= 21), after
// J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707 (2004):
// the coordinates are turned into the curve's "transposed" form by undoing
// the excess rotations/reflections level by level and Gray-coding, and the
// index is read off by interleaving the transposed bits, most significant
// level first, x before y before z.
uint64_t tm_hilbert3(uint32_t x, uint32_t y, uint32_t z, int bits) {
    uint32_t X[3] = {x, y, z};
    const uint32_t top = 1u << (bits - 1);
    for (uint32_t q = top; q > 1; q >>= 1) {
        const uint32_t low = q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & q) {
                X[0] ^= low;
            } else {
                const uint32_t t = (X[0] ^ X[i]) & low;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t flip = 0;
    for (uint32_t q = top; q > 1; q >>= 1)
        if (X[2] & q) flip ^= q - 1;
    for (int i = 0; i < 3; ++i) X[i] ^= flip;
    uint64_t key = 0;
    for (int b = bits - 1; b >= 0; --b)
        for (int i = 0; i < 3; ++i) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

namespace {

// Stable order of n items by key (ties by index).
void hilbert_order(const std::vector<uint64_t> &key, std::vector<int32_t> &perm) {
    const int64_t n = (int64_t)key.size();
    std::vector<std::pair<uint64_t, int32_t>> kv((size_t)n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) kv[(size_t)i] = {key[(size_t)i], (int32_t)i};
    __gnu_parallel::sort(kv.begin(), kv.end());
    perm.resize((size_t)n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = kv[(size_t)i].second;
}

// Concurrent union-find over tet ids: a root is a self-parent; union links
// the larger root below the smaller one with a compare-and-swap, find halves
// the path as it goes.  Used to label the regions of Sec. 5.
struct UnionFind {
    std::vector<std::atomic<int32_t>> parent;
    explicit UnionFind(int64_t n) : parent((size_t)n) {
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i) parent[(size_t)i].store((int32_t)i, std::memory_order_relaxed);
    }
    int32_t find(int32_t x) {
        for (;;) {
            int32_t p = parent[(size_t)x].load(std::memory_order_relaxed);
            if (p == x) return x;
            const int32_t g = parent[(size_t)p].load(std::memory_order_relaxed);
            if (g != p) parent[(size_t)x].compare_exchange_weak(p, g, std::memory_order_relaxed);
            x = g;
        }
    }
    void unite(int32_t a, int32_t b) {
        for (;;) {
            a = find(a);
            b = find(b);
            if (a == b) return;
            if (a < b) std::swap(a, b);
            int32_t expect = a;
            if (parent[(size_t)a].compare_exchange_strong(expect, b, std::memory_order_acq_rel)) return;
        }
    }
};

// Region of every tet (Sec. 5): 0..n_regions-1, numbered in the order of
// the smallest Hilbert key (key[t]) among their tets.
std::vector<int32_t> region_rank(const std::vector<uint32_t> &N, const std::vector<uint64_t> &key,
                                 int64_t nt) {
    UnionFind uf(nt);
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 4; ++k) {
            const uint32_t nb = N[(size_t)(4 * t + k)];
            if (!(nb & TM_CFACE_FLAG) && (int64_t)nb > t) uf.unite((int32_t)t, (int32_t)nb);
        }
    std::vector<int32_t> root((size_t)nt);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nt; ++t) root[(size_t)t] = uf.find((int32_t)t);
    // smallest key per root (roots are tet ids), then the roots in key order
    std::vector<uint64_t> kmin((size_t)nt, ~0ull);
    for (int64_t t = 0; t < nt; ++t) {
        uint64_t &k = kmin[(size_t)root[(size_t)t]];
        if (key[(size_t)t] < k) k = key[(size_t)t];
    }
    std::vector<std::pair<uint64_t, int32_t>> roots;
    for (int64_t t = 0; t < nt; ++t)
        if (root[(size_t)t] == t) roots.push_back({kmin[(size_t)t], (int32_t)t});
    std::sort(roots.begin(), roots.end());
    std::vector<int32_t> rank_of_root((size_t)nt, -1);
    for (size_t r = 0; r < roots.size(); ++r) rank_of_root[(size_t)roots[r].second] = (int32_t)r;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nt; ++t) root[(size_t)t] = rank_of_root[(size_t)root[(size_t)t]];
    return root;
}

inline uint32_t quantise(double v, double lo, double scale) {
    double q = std::floor((v - lo) * scale);
    if (q < 0) q = 0;
    if (q > 2097151.0) q = 2097151.0;
    return (uint32_t)q;
}

}  // namespace

tm_status tm_build_host(const float *points, int64_t np, const int32_t *tets_in, int64_t nt,
                        const int32_t *tris, int64_t nc, const tm_build_opts *opts, tm_mesh *m) {
    const int order = opts ? opts->order : TM_ORDER_HILBERT;
    const bool fix = opts ? opts->fix_orientation != 0 : false;
    const bool want_t20 = opts ? opts->tet20 != 0 : false;
    const bool want_face = opts ? opts->faces != 0 : false;
    const bool want_face16 = opts ? opts->faces16 != 0 : false;
    if (want_face16 && nt > (int64_t(1) << 29)) return TM_ERR_TOO_LARGE;  // tet ids share a word with w
    if (order != TM_ORDER_HILBERT && order != TM_ORDER_INPUT && order != TM_ORDER_HILBERT_REGIONS)
        return TM_ERR_ARG;
    m->np = np;
    m->nt = nt;
    m->nc = nc;

    // 1. ids and orientation -------------------------------------------------
    std::vector<int32_t> T((size_t)nt * 4);
    std::atomic<int> bad_range{0}, bad_orient{0};
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nt; ++t) {
        int32_t v[4];
        bool ok = true;
        for (int k = 0; k < 4; ++k) {
            v[k] = tets_in[4 * t + k];
            if (v[k] < 0 || v[k] >= np) ok = false;
        }
        if (!ok) { bad_range = 1; continue; }
        double P[4][3];
        for (int k = 0; k < 4; ++k)
            for (int a = 0; a < 3; ++a) P[k][a] = (double)points[3 * (int64_t)v[k] + a];
        const double o = orient3d(P[0], P[1], P[2], P[3]);
        if (!(o > 0.0)) {
            if (fix && o < 0.0) std::swap(v[2], v[3]);
            else bad_orient = 1;
        }
        for (int k = 0; k < 4; ++k) T[(size_t)(4 * t + k)] = v[k];
    }
    if (bad_range) return TM_ERR_RANGE;
    for (int64_t i = 0; i < 3 * nc; ++i)
        if (tris[i] < 0 || tris[i] >= np) return TM_ERR_RANGE;
    if (bad_orient) return TM_ERR_ORIENT;

    // 2. neighbours by min-vertex buckets -------------------------------------
    std::vector<int64_t> start((size_t)np + 1, 0);
    {
        std::vector<std::atomic<int32_t>> cnt((size_t)np);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < np; ++i) cnt[(size_t)i].store(0, std::memory_order_relaxed);
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < nt; ++t)
            for (int k = 0; k < 4; ++k) {
                int32_t a = T[4 * t + kFaceIn[k][0]], b = T[4 * t + kFaceIn[k][1]],
                        c = T[4 * t + kFaceIn[k][2]];
                sort3(a, b, c);
                cnt[(size_t)a].fetch_add(1, std::memory_order_relaxed);
            }
        for (int64_t i = 0; i < np; ++i) start[(size_t)i + 1] = start[(size_t)i] + cnt[(size_t)i].load();
    }
    std::vector<FaceEntry> F((size_t)(4 * nt));
    {
        std::vector<std::atomic<int64_t>> cur((size_t)np);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < np; ++i) cur[(size_t)i].store(start[(size_t)i], std::memory_order_relaxed);
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < nt; ++t)
            for (int k = 0; k < 4; ++k) {
                int32_t a = T[4 * t + kFaceIn[k][0]], b = T[4 * t + kFaceIn[k][1]],
                        c = T[4 * t + kFaceIn[k][2]];
                sort3(a, b, c);
                const int64_t pos = cur[(size_t)a].fetch_add(1, std::memory_order_relaxed);
                F[(size_t)pos] = FaceEntry{b, c, (int32_t)(4 * t + k)};
            }
    }
    std::vector<uint32_t> N((size_t)nt * 4, TM_BOUNDARY);
    std::atomic<int> nonmanifold{0};
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t a = 0; a < np; ++a) {
        FaceEntry *lo = F.data() + start[(size_t)a], *hi = F.data() + start[(size_t)a + 1];
        std::sort(lo, hi, face_less);
        for (FaceEntry *p = lo; p < hi;) {
            FaceEntry *q = p + 1;
            while (q < hi && q->b == p->b && q->c == p->c) ++q;
            if (q - p > 2) nonmanifold = 1;
            else if (q - p == 2) {
                N[(size_t)p[0].owner] = (uint32_t)(p[1].owner >> 2);
                N[(size_t)p[1].owner] = (uint32_t)(p[0].owner >> 2);
            }
            p = q;
        }
    }
    if (nonmanifold) return TM_ERR_NONMANIFOLD;

    // 3. constrained faces --------------------------------------------------------
    std::vector<int32_t> ctet((size_t)nc * 2, -1);
    std::atomic<int> unmatched{0}, duplicate{0};
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        int32_t a = tris[3 * c], b = tris[3 * c + 1], d = tris[3 * c + 2];
        sort3(a, b, d);
        const FaceEntry *lo = F.data() + start[(size_t)a], *hi = F.data() + start[(size_t)a + 1];
        const FaceEntry key{b, d, -1};
        const FaceEntry *p = std::lower_bound(lo, hi, key, face_less);
        if (p == hi || p->b != b || p->c != d) { unmatched = 1; continue; }
        double V[3][3];
        for (int i = 0; i < 3; ++i)
            for (int x = 0; x < 3; ++x) V[i][x] = (double)points[3 * (int64_t)tris[3 * c + i] + x];
        for (; p < hi && p->b == b && p->c == d; ++p) {
            const int32_t t = p->owner >> 2, k = p->owner & 3;
            double X[3];
            for (int x = 0; x < 3; ++x) X[x] = (double)points[3 * (int64_t)T[4 * t + k] + x];
            const int side = orient3d(V[0], V[1], V[2], X) > 0.0 ? 0 : 1;
            if (ctet[2 * c + side] >= 0) duplicate = 1;
            ctet[2 * c + side] = t;
        }
    }
    if (unmatched) return TM_ERR_CFACE_UNMATCHED;
    if (duplicate) return TM_ERR_CFACE_DUPLICATE;
    // flag the neighbour fields (two triangles on one face is an error)
    std::vector<std::atomic<uint8_t>> used((size_t)nt * 4);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < 4 * nt; ++i) used[(size_t)i].store(0, std::memory_order_relaxed);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        for (int s = 0; s < 2; ++s) {
            const int32_t t = ctet[2 * c + s];
            if (t < 0) continue;
            int32_t a = tris[3 * c], b = tris[3 * c + 1], d = tris[3 * c + 2];
            sort3(a, b, d);
            for (int k = 0; k < 4; ++k) {
                int32_t x = T[4 * t + kFaceIn[k][0]], y = T[4 * t + kFaceIn[k][1]],
                        z = T[4 * t + kFaceIn[k][2]];
                sort3(x, y, z);
                if (x == a && y == b && z == d) {
                    if (used[(size_t)(4 * t + k)].exchange(1)) duplicate = 1;
                    N[(size_t)(4 * t + k)] = TM_CFACE_FLAG | (uint32_t)c;
                }
            }
        }
    }
    if (duplicate) return TM_ERR_CFACE_DUPLICATE;
    F.clear();
    F.shrink_to_fit();

    // bounding box / extent
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < np; ++i)
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], (double)points[3 * i + a]);
            hi[a] = std::max(hi[a], (double)points[3 * i + a]);
        }
    m->extent = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    for (int a = 0; a < 3; ++a) { m->lo[a] = (float)lo[a]; m->hi[a] = (float)hi[a]; }

    // 4. Hilbert order --------------------------------------------------------------
    m->pperm.resize((size_t)np);
    m->tperm.resize((size_t)nt);
    if (order == TM_ORDER_HILBERT || order == TM_ORDER_HILBERT_REGIONS) {
        const double span = m->extent > 0 ? m->extent : 1.0;
        const double scale = 2097152.0 / span;
        std::vector<uint64_t> key((size_t)np);
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < np; ++i)
            key[(size_t)i] = tm_hilbert3(quantise(points[3 * i], lo[0], scale),
                                         quantise(points[3 * i + 1], lo[1], scale),
                                         quantise(points[3 * i + 2], lo[2], scale), 21);
        hilbert_order(key, m->pperm);
        key.assign((size_t)nt, 0);
#pragma omp parallel for schedule(static)
        for (int64_t t = 0; t < nt; ++t) {
            double c[3] = {0, 0, 0};
            for (int k = 0; k < 4; ++k)
                for (int a = 0; a < 3; ++a) c[a] += (double)points[3 * (int64_t)T[4 * t + k] + a];
            key[(size_t)t] = tm_hilbert3(quantise(0.25 * c[0], lo[0], scale),
                                         quantise(0.25 * c[1], lo[1], scale),
                                         quantise(0.25 * c[2], lo[2], scale), 21);
        }
        if (order == TM_ORDER_HILBERT_REGIONS) {
            // tets sorted by (region, Hilbert key, input id)
            const std::vector<int32_t> reg = region_rank(N, key, nt);
            std::vector<std::pair<std::pair<int32_t, uint64_t>, int32_t>> kv((size_t)nt);
#pragma omp parallel for schedule(static)
            for (int64_t t = 0; t < nt; ++t) kv[(size_t)t] = {{reg[(size_t)t], key[(size_t)t]}, (int32_t)t};
            __gnu_parallel::sort(kv.begin(), kv.end());
#pragma omp parallel for schedule(static)
            for (int64_t t = 0; t < nt; ++t) m->tperm[(size_t)t] = kv[(size_t)t].second;
            int32_t nreg = 0;
            for (int64_t t = 0; t < nt; ++t) nreg = std::max(nreg, reg[(size_t)t] + 1);
            m->n_regions = nreg;
        } else {
            hilbert_order(key, m->tperm);
        }
    } else {
        for (int64_t i = 0; i < np; ++i) m->pperm[(size_t)i] = (int32_t)i;
        for (int64_t t = 0; t < nt; ++t) m->tperm[(size_t)t] = (int32_t)t;
    }
    m->pinv.resize((size_t)np);
    m->tinv.resize((size_t)nt);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < np; ++i) m->pinv[(size_t)m->pperm[(size_t)i]] = (int32_t)i;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nt; ++t) m->tinv[(size_t)m->tperm[(size_t)t]] = (int32_t)t;

    // 5. packing ----------------------------------------------------------------------
    m->pts4.resize((size_t)np * 4);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < np; ++i) {
        const int64_t o = m->pperm[(size_t)i];
        m->pts4[4 * i + 0] = points[3 * o + 0];
        m->pts4[4 * i + 1] = points[3 * o + 1];
        m->pts4[4 * i + 2] = points[3 * o + 2];
        m->pts4[4 * i + 3] = 0.0f;
    }
    m->cold.resize((size_t)nt * 8);
    m->tet16.resize((size_t)nt * 4);
    if (want_t20) {
        m->t20.resize((size_t)nt * 4);
        m->t20n3.resize((size_t)nt);
        m->t20aos.resize((size_t)nt * 5);
    }
#pragma omp parallel for schedule(static)
    for (int64_t tn = 0; tn < nt; ++tn) {
        const int64_t t = m->tperm[(size_t)tn];
        int32_t V[4];
        uint32_t NB[4];
        for (int k = 0; k < 4; ++k) {
            V[k] = m->pinv[(size_t)T[4 * t + k]];
            const uint32_t raw = N[(size_t)(4 * t + k)];
            NB[k] = (raw & TM_CFACE_FLAG) ? raw : (uint32_t)m->tinv[raw];
            m->cold[8 * tn + k] = V[k];
            m->cold[8 * tn + 4 + k] = (int32_t)NB[k];
        }
        // neighbours sorted by the id of the vertex they sit across
        int idx[4] = {0, 1, 2, 3};
        std::sort(idx, idx + 4, [&](int x, int y) { return V[x] < V[y]; });
        const uint32_t n3 = NB[idx[3]];
        m->tet16[4 * tn + 0] = V[0] ^ V[1] ^ V[2] ^ V[3];
        m->tet16[4 * tn + 1] = (int32_t)(NB[idx[0]] ^ n3);
        m->tet16[4 * tn + 2] = (int32_t)(NB[idx[1]] ^ n3);
        m->tet16[4 * tn + 3] = (int32_t)(NB[idx[2]] ^ n3);
        if (want_t20) {
            m->t20[4 * tn + 0] = m->tet16[4 * tn + 0];
            m->t20[4 * tn + 1] = (int32_t)NB[idx[0]];
            m->t20[4 * tn + 2] = (int32_t)NB[idx[1]];
            m->t20[4 * tn + 3] = (int32_t)NB[idx[2]];
            m->t20n3[tn] = (int32_t)n3;
            for (int j = 0; j < 4; ++j) m->t20aos[5 * tn + j] = m->t20[4 * tn + j];
            m->t20aos[5 * tn + 4] = (int32_t)n3;
        }
    }
    if (want_face) {
        // face entry r of tet T: the face opposite T's vertex of rank r; the
        // neighbour N across it and N's vertex opposite the shared face
        m->face.assign((size_t)nt * 32, 0);
#pragma omp parallel for schedule(static)
        for (int64_t tn = 0; tn < nt; ++tn) {
            const int32_t *V = &m->cold[8 * tn];
            const int32_t *NB = &m->cold[8 * tn + 4];
            int idx[4] = {0, 1, 2, 3};
            std::sort(idx, idx + 4, [&](int x, int y) { return V[x] < V[y]; });
            for (int r = 0; r < 4; ++r) {
                int32_t *e = &m->face[32 * tn + 8 * r];
                const uint32_t nb = (uint32_t)NB[idx[r]];
                e[0] = (int32_t)nb;
                e[1] = -1;
                if (nb & TM_CFACE_FLAG) continue;
                const int32_t *V2 = &m->cold[8 * (int64_t)nb];
                const int32_t *N2 = &m->cold[8 * (int64_t)nb + 4];
                for (int j = 0; j < 4; ++j)
                    if (N2[j] == (int32_t)tn) {
                        e[1] = V2[j];
                        std::memcpy(&e[2], &m->pts4[4 * (int64_t)V2[j]], 3 * sizeof(float));
                    }
            }
        }
    }
    if (want_face16) {
        // entry r of tet T: the neighbour N across the face opposite T's
        // vertex of rank r, the rank w of N's opposite vertex W among N's
        // vertex ids (bits 29-30), and W's position
        m->face16.assign((size_t)nt * 16, 0);
#pragma omp parallel for schedule(static)
        for (int64_t tn = 0; tn < nt; ++tn) {
            const int32_t *V = &m->cold[8 * tn];
            const int32_t *NB = &m->cold[8 * tn + 4];
            int idx[4] = {0, 1, 2, 3};
            std::sort(idx, idx + 4, [&](int x, int y) { return V[x] < V[y]; });
            for (int r = 0; r < 4; ++r) {
                int32_t *e = &m->face16[16 * tn + 4 * r];
                const uint32_t nb = (uint32_t)NB[idx[r]];
                e[0] = (int32_t)nb;
                if (nb & TM_CFACE_FLAG) continue;
                const int32_t *V2 = &m->cold[8 * (int64_t)nb];
                const int32_t *N2 = &m->cold[8 * (int64_t)nb + 4];
                for (int j = 0; j < 4; ++j)
                    if (N2[j] == (int32_t)tn) {
                        const int32_t w = V2[j];
                        const uint32_t wr = (uint32_t)((V2[0] < w) + (V2[1] < w) + (V2[2] < w) + (V2[3] < w));
                        e[0] = (int32_t)(nb | (wr << 29));
                        std::memcpy(&e[1], &m->pts4[4 * (int64_t)w], 3 * sizeof(float));
                    }
            }
        }
    }
    m->cface.resize((size_t)nc * 8);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        int32_t *r = &m->cface[8 * c];
        r[0] = (int32_t)c;
        r[1] = ctet[2 * c] >= 0 ? m->tinv[(size_t)ctet[2 * c]] : -1;
        r[2] = ctet[2 * c + 1] >= 0 ? m->tinv[(size_t)ctet[2 * c + 1]] : -1;
        r[3] = 0;
        r[4] = m->pinv[(size_t)tris[3 * c]];
        r[5] = m->pinv[(size_t)tris[3 * c + 1]];
        r[6] = m->pinv[(size_t)tris[3 * c + 2]];
        r[7] = 0;
    }
    // the hit kernels' view of a triangle: its three vertices inline (one
    // 48-byte read instead of the record and three point reads)
    m->cgeo.resize((size_t)nc * 12);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        int32_t *g = &m->cgeo[12 * c];
        for (int k = 0; k < 3; ++k)
            std::memcpy(&g[4 * k], &m->pts4[4 * (int64_t)m->cface[8 * c + 4 + k]], 3 * sizeof(float));
        g[3] = m->cface[8 * c + 1];
        g[7] = (int32_t)c;
        g[11] = 0;
    }
    // restart records: for side s of triangle c, the tet on that side (its
    // cold record, its vertices' positions, and the local index of the face
    // it shares with c), so that a restarted ray needs one read to start
    m->restart.assign((size_t)nc * 2 * 24, 0);
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < nc; ++c) {
        for (int side = 0; side < 2; ++side) {
            int32_t *r = &m->restart[24 * (2 * c + side)];
            const int32_t T = m->cface[8 * c + 1 + side];
            r[20] = -1;
            r[21] = -1;
            if (T < 0) continue;
            const int32_t *V = &m->cold[8 * (int64_t)T];
            const int32_t *N = &m->cold[8 * (int64_t)T + 4];
            int skip = -1;
            for (int k = 0; k < 4; ++k)
                if ((uint32_t)N[k] == (TM_CFACE_FLAG | (uint32_t)c)) skip = k;
            for (int k = 0; k < 4; ++k) {
                r[k] = V[k];
                r[4 + k] = N[k];
                std::memcpy(&r[8 + 3 * k], &m->pts4[4 * (int64_t)V[k]], 3 * sizeof(float));
            }
            r[20] = T;
            r[21] = skip;
        }
    }

    // default locate source: the tet whose centroid is nearest the box centre
    const double cen[3] = {0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2])};
    double best = INFINITY;
    int32_t best_t = 0;
#pragma omp parallel
    {
        double lb = INFINITY;
        int32_t lt = 0;
#pragma omp for schedule(static) nowait
        for (int64_t tn = 0; tn < nt; ++tn) {
            double c[3] = {0, 0, 0};
            for (int k = 0; k < 4; ++k)
                for (int a = 0; a < 3; ++a) c[a] += m->pts4[4 * (int64_t)m->cold[8 * tn + k] + a];
            double d2 = 0;
            for (int a = 0; a < 3; ++a) d2 += (0.25 * c[a] - cen[a]) * (0.25 * c[a] - cen[a]);
            if (d2 < lb) { lb = d2; lt = (int32_t)tn; }
        }
#pragma omp critical
        {
            if (lb < best || (lb == best && lt < best_t)) { best = lb; best_t = lt; }
        }
    }
    m->source_tet = best_t;
    return TM_OK;
}

tm_status tm_upload(tm_mesh *m) {
    TM_CUDA(cudaGetDevice(&m->device));
    const size_t b_tet = sizeof(int4) * (size_t)m->nt, b_pts = sizeof(float4) * (size_t)m->np,
                 b_cold = 2 * sizeof(int4) * (size_t)m->nt,
                 b_cf = 2 * sizeof(int4) * (size_t)(m->nc > 0 ? m->nc : 1),
                 b_cg = 3 * sizeof(int4) * (size_t)(m->nc > 0 ? m->nc : 1),
                 b_rs = 12 * sizeof(int4) * (size_t)(m->nc > 0 ? m->nc : 1);
    cudaError_t e;
    if ((e = cudaMalloc(&m->d_tet16, b_tet)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_pts, b_pts)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_cold, b_cold)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_cface, b_cf)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_cgeo, b_cg)) != cudaSuccess ||
        (e = cudaMalloc(&m->d_restart, b_rs)) != cudaSuccess) {
        tm_set_error("cudaMalloc", e);
        return e == cudaErrorMemoryAllocation ? TM_ERR_OOM : TM_ERR_CUDA;
    }
    TM_CUDA(cudaMemcpy(m->d_tet16, m->tet16.data(), b_tet, cudaMemcpyHostToDevice));
    TM_CUDA(cudaMemcpy(m->d_pts, m->pts4.data(), b_pts, cudaMemcpyHostToDevice));
    TM_CUDA(cudaMemcpy(m->d_cold, m->cold.data(), b_cold, cudaMemcpyHostToDevice));
    if (m->nc > 0)
        TM_CUDA(cudaMemcpy(m->d_cface, m->cface.data(), 2 * sizeof(int4) * (size_t)m->nc,
                           cudaMemcpyHostToDevice));
    if (m->nc > 0) {
        TM_CUDA(cudaMemcpy(m->d_cgeo, m->cgeo.data(), 3 * sizeof(int4) * (size_t)m->nc,
                           cudaMemcpyHostToDevice));
        TM_CUDA(cudaMemcpy(m->d_restart, m->restart.data(), 12 * sizeof(int4) * (size_t)m->nc,
                           cudaMemcpyHostToDevice));
    }
    m->device_bytes = (int64_t)(b_tet + b_pts + b_cold + b_cf + b_cg + b_rs);
    if (!m->t20.empty()) {
        TM_CUDA(cudaMalloc(&m->d_t20, sizeof(int4) * (size_t)m->nt));
        TM_CUDA(cudaMalloc(&m->d_t20n3, sizeof(int32_t) * (size_t)m->nt));
        TM_CUDA(cudaMemcpy(m->d_t20, m->t20.data(), sizeof(int4) * (size_t)m->nt, cudaMemcpyHostToDevice));
        TM_CUDA(cudaMemcpy(m->d_t20n3, m->t20n3.data(), sizeof(int32_t) * (size_t)m->nt,
                           cudaMemcpyHostToDevice));
        TM_CUDA(cudaMalloc(&m->d_t20aos, 5 * sizeof(int32_t) * (size_t)m->nt));
        TM_CUDA(cudaMemcpy(m->d_t20aos, m->t20aos.data(), 5 * sizeof(int32_t) * (size_t)m->nt,
                           cudaMemcpyHostToDevice));
        m->device_bytes += (int64_t)(40 * m->nt);
    }
    if (!m->face16.empty()) {
        TM_CUDA(cudaMalloc(&m->d_face16, 64 * (size_t)m->nt));
        TM_CUDA(cudaMemcpy(m->d_face16, m->face16.data(), 64 * (size_t)m->nt, cudaMemcpyHostToDevice));
        m->device_bytes += (int64_t)(64 * m->nt);
    }
    if (!m->face.empty()) {
        TM_CUDA(cudaMalloc(&m->d_face, 128 * (size_t)m->nt));
        TM_CUDA(cudaMemcpy(m->d_face, m->face.data(), 128 * (size_t)m->nt, cudaMemcpyHostToDevice));
        m->device_bytes += (int64_t)(128 * m->nt);
    }
    m->on_device = true;
    // seed lattice: locate the centres of a kSeedGrid^3 lattice over the
    // bounding cube once, from the default source tet
    const int G = kSeedGrid, ns = G * G * G;
    std::vector<float> q((size_t)ns * 3);
    for (int k = 0; k < G; ++k)
        for (int j = 0; j < G; ++j)
            for (int i = 0; i < G; ++i) {
                const size_t c = (size_t)(i + G * (j + G * k));
                q[3 * c + 0] = (float)(m->lo[0] + (i + 0.5) * m->extent / G);
                q[3 * c + 1] = (float)(m->lo[1] + (j + 0.5) * m->extent / G);
                q[3 * c + 2] = (float)(m->lo[2] + (k + 0.5) * m->extent / G);
            }
    float *d_q = nullptr;
    TM_CUDA(cudaMalloc(&m->d_seeds, sizeof(int32_t) * ns));
    TM_CUDA(cudaMalloc(&d_q, sizeof(float) * 3 * ns));
    const cudaError_t ec = cudaMemcpy(d_q, q.data(), sizeof(float) * 3 * ns, cudaMemcpyHostToDevice);
    if (ec != cudaSuccess) {
        cudaFree(d_q);
        tm_set_error("cudaMemcpy (seed lattice)", ec);
        return TM_ERR_CUDA;
    }
    MeshView mv = mesh_view(m);
    mv.seeds = nullptr;  // the lattice itself is located from the default source
    const uint32_t bound = (uint32_t)(64.0 * std::cbrt((double)m->nt) * 8.0 + 1024.0);
    tm_status st = launch_locate(mv, d_q, ns, nullptr, m->source_tet, m->d_seeds, bound, 0);
    cudaError_t e2 = cudaDeviceSynchronize();
    cudaFree(d_q);
    if (st != TM_OK) return st;
    if (e2 != cudaSuccess) {
        tm_set_error("seed lattice", e2);
        return TM_ERR_CUDA;
    }
    m->device_bytes += (int64_t)(sizeof(int32_t) * ns);
    return TM_OK;
}

void tm_free_device(tm_mesh *m) {
    if (!m->on_device && !m->d_tet16 && !m->d_pts && !m->d_cold && !m->d_cface) return;
    int cur = -1;
    cudaGetDevice(&cur);
    if (m->device >= 0 && m->device != cur) cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    cudaFree(m->d_tet16);
    cudaFree(m->d_pts);
    cudaFree(m->d_cold);
    cudaFree(m->d_cface);
    cudaFree(m->d_cgeo);
    m->d_cgeo = nullptr;
    cudaFree(m->d_restart);
    m->d_restart = nullptr;
    cudaFree(m->d_seeds);
    m->d_seeds = nullptr;
    cudaFree(m->d_t20);
    cudaFree(m->d_t20n3);
    cudaFree(m->d_t20aos);
    cudaFree(m->d_face);
    m->d_face = nullptr;
    cudaFree(m->d_face16);
    m->d_face16 = nullptr;
    m->d_t20 = nullptr;
    m->d_t20n3 = nullptr;
    m->d_t20aos = nullptr;
    m->d_tet16 = nullptr;
    m->d_pts = nullptr;
    m->d_cold = nullptr;
    m->d_cface = nullptr;
    m->on_device = false;
    if (m->device >= 0 && m->device != cur && cur >= 0) cudaSetDevice(cur);
}
