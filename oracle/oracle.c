/*
 * oracle.c -- plain, slow FP64 reference for ray traversal of a constrained
 * tetrahedral mesh.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls
 * it.
 *
 * What it computes is the plain definition of the traversal result
 * (Sec. 4 and Sec. 6 of the paper: a ray walks face-adjacent tetrahedra from
 * the tet that holds its origin and stops at the first constrained face or at
 * the mesh boundary):
 *
 *   x(t) = o + t d, with o, d, t_max the float32 inputs promoted exactly to
 *   double.  The hit is the constrained triangle (closed, two-sided) with the
 *   smallest t in (0, t_max]; a ray restarted from a constrained face excludes
 *   that face.  Output: triangle row id, t, and (b1, b2) with
 *   x = (1-b1-b2) v0 + b1 v1 + b2 v2 in the triangle's own vertex order.
 *   A ray that leaves the mesh first, or hits nothing before t_max, misses.
 *
 * Two independent ways to reach it are provided:
 *   orc_trace      -- a 3-D "closest exit face" walk (the face-plane method of
 *                     Garrity 1990, cited in Sec. 2.2 of the paper): in each
 *                     tet, intersect the ray with the planes of the faces it
 *                     can leave through and take the nearest one.
 *   orc_bruteforce -- Moller-Trumbore (1997) against every constrained
 *                     triangle, nearest t.
 * plus orc_locate (brute force point-in-tet, Sec. 4.2's operation) and the
 * mesh invariant checkers (positive orientation, symmetric neighbours,
 * constrained faces matched to tet faces).
 *
 * Conventions: a tet (V0,V1,V2,V3) is positively oriented when
 * orient3d(V0,V1,V2,V3) = det[V1-V0, V2-V0, V3-V0] > 0.  Local face k is the
 * face opposite V_k.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_FLAG_STEP_LIMIT 1
#define ORC_FLAG_DEGENERATE 2   /* no face with an exiting plane */
#define ORC_FLAG_BAD_START 4    /* restart face not found / no tet on that side */
#define ORC_FLAG_NONMONOTONE 8  /* exit t decreased: a broken walk */
#define ORC_FLAG_TIE 16         /* two consecutive exits at equal t (ray through an edge/vertex) */

/* Vertex slots of local face k (opposite V_k), in the order whose normal
 * (b-a) x (c-a) points into a positively oriented tet. */
static const int FACE[4][3] = {{1, 3, 2}, {0, 2, 3}, {0, 3, 1}, {0, 1, 2}};

typedef struct orc_mesh {
    int64_t np, nt, nc;
    double *P;      /* np*3 point coordinates */
    int32_t *T;     /* nt*4 vertex ids */
    int32_t *tri;   /* nc*3 triangle vertex ids */
    int32_t *nbr;   /* nt*4 neighbour across face k, -1 on the boundary */
    int32_t *nbrk;  /* nt*4 local index of the same face in that neighbour */
    int32_t *fc;    /* nt*4 constrained triangle lying on face k, or -1 */
    int32_t *ctet;  /* nc*2 tet on the + and - side of each triangle (-1 none) */
} orc_mesh;

static void sub3(const double *a, const double *b, double *r) {
    r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2];
}
static void cross3(const double *a, const double *b, double *r) {
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static double orient3d(const double *a, const double *b, const double *c, const double *d) {
    double ab[3], ac[3], ad[3], n[3];
    sub3(b, a, ab); sub3(c, a, ac); sub3(d, a, ad);
    cross3(ab, ac, n);
    return dot3(n, ad);
}

/* ------------------------------------------------------------------------ */
/* Adjacency by sorting the vertex triples of all 4*nt faces.                */

typedef struct { int32_t a, b, c; int32_t owner; } face_rec; /* owner = 4*tet + k */

static void sort3(int32_t *x, int32_t *y, int32_t *z) {
    int32_t t;
    if (*x > *y) { t = *x; *x = *y; *y = t; }
    if (*y > *z) { t = *y; *y = *z; *z = t; }
    if (*x > *y) { t = *x; *x = *y; *y = t; }
}
static int cmp_face(const void *pa, const void *pb) {
    const face_rec *a = (const face_rec *)pa, *b = (const face_rec *)pb;
    if (a->a != b->a) return a->a < b->a ? -1 : 1;
    if (a->b != b->b) return a->b < b->b ? -1 : 1;
    if (a->c != b->c) return a->c < b->c ? -1 : 1;
    return a->owner < b->owner ? -1 : (a->owner > b->owner);
}
static int find_face(const face_rec *F, int64_t nf, int32_t a, int32_t b, int32_t c) {
    int64_t lo = 0, hi = nf;
    face_rec key = {a, b, c, -1};
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (cmp_face(&F[mid], &key) < 0) lo = mid + 1; else hi = mid;
    }
    return (int)(lo < nf && F[lo].a == a && F[lo].b == b && F[lo].c == c) ? 1 : 0;
}
static int64_t lower_face(const face_rec *F, int64_t nf, int32_t a, int32_t b, int32_t c) {
    int64_t lo = 0, hi = nf;
    face_rec key = {a, b, c, -1};
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        if (cmp_face(&F[mid], &key) < 0) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Status: 0 ok, 1 bad argument / id out of range, 2 a face shared by more
 * than two tets, 3 a triangle that is no tet face, 4 two triangles on one
 * face, 5 out of memory. */
int orc_mesh_create(int64_t np, const float *pts, int64_t nt, const int32_t *tets,
                    int64_t nc, const int32_t *tris, orc_mesh **out) {
    *out = NULL;
    if (np <= 0 || nt <= 0 || nc < 0) return 1;
    orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
    if (!m) return 5;
    m->np = np; m->nt = nt; m->nc = nc;
    m->P = (double *)malloc(sizeof(double) * 3 * np);
    m->T = (int32_t *)malloc(sizeof(int32_t) * 4 * nt);
    m->tri = (int32_t *)malloc(sizeof(int32_t) * 3 * (nc > 0 ? nc : 1));
    m->nbr = (int32_t *)malloc(sizeof(int32_t) * 4 * nt);
    m->nbrk = (int32_t *)malloc(sizeof(int32_t) * 4 * nt);
    m->fc = (int32_t *)malloc(sizeof(int32_t) * 4 * nt);
    m->ctet = (int32_t *)malloc(sizeof(int32_t) * 2 * (nc > 0 ? nc : 1));
    face_rec *F = (face_rec *)malloc(sizeof(face_rec) * 4 * nt);
    int status = 0;
    if (!m->P || !m->T || !m->tri || !m->nbr || !m->nbrk || !m->fc || !m->ctet || !F) {
        status = 5; goto fail;
    }
    for (int64_t i = 0; i < 3 * np; ++i) m->P[i] = (double)pts[i];
    memcpy(m->T, tets, sizeof(int32_t) * 4 * nt);
    if (nc > 0) memcpy(m->tri, tris, sizeof(int32_t) * 3 * nc);
    for (int64_t i = 0; i < 4 * nt; ++i) {
        if (tets[i] < 0 || tets[i] >= np) { status = 1; goto fail; }
        m->nbr[i] = -1; m->nbrk[i] = -1; m->fc[i] = -1;
    }
    for (int64_t i = 0; i < 3 * nc; ++i)
        if (tris[i] < 0 || tris[i] >= np) { status = 1; goto fail; }

    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 4; ++k) {
            face_rec *f = &F[4 * t + k];
            f->a = tets[4 * t + FACE[k][0]];
            f->b = tets[4 * t + FACE[k][1]];
            f->c = tets[4 * t + FACE[k][2]];
            sort3(&f->a, &f->b, &f->c);
            f->owner = (int32_t)(4 * t + k);
        }
    qsort(F, (size_t)(4 * nt), sizeof(face_rec), cmp_face);
    for (int64_t i = 0; i < 4 * nt;) {
        int64_t j = i + 1;
        while (j < 4 * nt && F[j].a == F[i].a && F[j].b == F[i].b && F[j].c == F[i].c) ++j;
        if (j - i > 2) { status = 2; goto fail; }
        if (j - i == 2) {
            int32_t o0 = F[i].owner, o1 = F[i + 1].owner;
            m->nbr[o0] = o1 / 4; m->nbrk[o0] = o1 % 4;
            m->nbr[o1] = o0 / 4; m->nbrk[o1] = o0 % 4;
        }
        i = j;
    }
    for (int64_t c = 0; c < nc; ++c) {
        int32_t a = tris[3 * c], b = tris[3 * c + 1], d = tris[3 * c + 2];
        sort3(&a, &b, &d);
        if (!find_face(F, 4 * nt, a, b, d)) { status = 3; goto fail; }
        m->ctet[2 * c] = -1; m->ctet[2 * c + 1] = -1;
        const double *v0 = m->P + 3 * tris[3 * c], *v1 = m->P + 3 * tris[3 * c + 1],
                     *v2 = m->P + 3 * tris[3 * c + 2];
        for (int64_t i = lower_face(F, 4 * nt, a, b, d);
             i < 4 * nt && F[i].a == a && F[i].b == b && F[i].c == d; ++i) {
            int32_t o = F[i].owner;
            if (m->fc[o] >= 0) { status = 4; goto fail; }
            m->fc[o] = (int32_t)c;
            /* side of the tet: sign of its opposite vertex against the
             * triangle's own plane (normal (v1-v0) x (v2-v0)). */
            int32_t t = o / 4, k = o % 4;
            double s = orient3d(v0, v1, v2, m->P + 3 * tets[4 * t + k]);
            m->ctet[2 * c + (s > 0 ? 0 : 1)] = t;
        }
    }
    free(F);
    *out = m;
    return 0;
fail:
    free(F);
    free(m->P); free(m->T); free(m->tri); free(m->nbr); free(m->nbrk); free(m->fc); free(m->ctet);
    free(m);
    return status;
}

void orc_mesh_destroy(orc_mesh *m);

/* A triangle set without tets: points and constrained triangles only, for
 * orc_bruteforce on scenes too large for the adjacency build (no walk,
 * location or checker may be called on it).  Status as orc_mesh_create. */
int orc_soup_create(int64_t np, const float *pts, int64_t nc, const int32_t *tris,
                    orc_mesh **out) {
    *out = NULL;
    if (np <= 0 || nc < 0) return 1;
    orc_mesh *m = (orc_mesh *)calloc(1, sizeof(orc_mesh));
    if (!m) return 5;
    m->np = np; m->nc = nc;
    m->P = (double *)malloc(sizeof(double) * 3 * np);
    m->tri = (int32_t *)malloc(sizeof(int32_t) * 3 * (nc > 0 ? nc : 1));
    if (!m->P || !m->tri) { orc_mesh_destroy(m); return 5; }
    for (int64_t i = 0; i < 3 * np; ++i) m->P[i] = (double)pts[i];
    for (int64_t i = 0; i < 3 * nc; ++i) {
        if (tris[i] < 0 || tris[i] >= np) { orc_mesh_destroy(m); return 1; }
        m->tri[i] = tris[i];
    }
    *out = m;
    return 0;
}

void orc_mesh_destroy(orc_mesh *m) {
    if (!m) return;
    free(m->P); free(m->T); free(m->tri); free(m->nbr); free(m->nbrk); free(m->fc); free(m->ctet);
    free(m);
}

/* Copies the oracle's adjacency: neighbour tet across face k (-1 boundary),
 * the constrained triangle on face k (-1 none), and per triangle the tets on
 * its + and - side. */
void orc_mesh_arrays(const orc_mesh *m, int32_t *nbr, int32_t *fc, int32_t *ctet) {
    if (nbr) memcpy(nbr, m->nbr, sizeof(int32_t) * 4 * m->nt);
    if (fc) memcpy(fc, m->fc, sizeof(int32_t) * 4 * m->nt);
    if (ctet && m->nc > 0) memcpy(ctet, m->ctet, sizeof(int32_t) * 2 * m->nc);
}

/* ------------------------------------------------------------------------ */
/* Invariant checkers.                                                       */

/* Number of tets with orient3d <= 0. */
int64_t orc_count_nonpositive(const orc_mesh *m) {
    int64_t bad = 0;
    for (int64_t t = 0; t < m->nt; ++t) {
        const int32_t *v = m->T + 4 * t;
        if (!(orient3d(m->P + 3 * v[0], m->P + 3 * v[1], m->P + 3 * v[2], m->P + 3 * v[3]) > 0)) ++bad;
    }
    return bad;
}

/* Number of (tet, face) pairs whose neighbour does not point back through a
 * face with the same three vertices. */
int64_t orc_count_asymmetric(const orc_mesh *m) {
    int64_t bad = 0;
    for (int64_t t = 0; t < m->nt; ++t)
        for (int k = 0; k < 4; ++k) {
            int32_t u = m->nbr[4 * t + k];
            if (u < 0) continue;
            int32_t ku = m->nbrk[4 * t + k];
            if (m->nbr[4 * u + ku] != t) { ++bad; continue; }
            int32_t a = m->T[4 * t + FACE[k][0]], b = m->T[4 * t + FACE[k][1]], c = m->T[4 * t + FACE[k][2]];
            int32_t x = m->T[4 * u + FACE[ku][0]], y = m->T[4 * u + FACE[ku][1]], z = m->T[4 * u + FACE[ku][2]];
            sort3(&a, &b, &c); sort3(&x, &y, &z);
            if (a != x || b != y || c != z) ++bad;
        }
    return bad;
}

/* Test hook for the checkers' pins: overwrites the link of tet t across its
 * face k with (u, ku), the neighbour and the index of the shared face inside
 * it (u = -1 for the boundary), so that a test can plant a broken adjacency
 * and see orc_count_asymmetric report it.  Returns 1 on bad arguments. */
int orc_mesh_relink(orc_mesh *m, int64_t t, int k, int32_t u, int ku) {
    if (!m || !m->nbr || t < 0 || t >= m->nt || k < 0 || k > 3 || u < -1 || u >= m->nt ||
        ku < -1 || ku > 3)
        return 1;
    m->nbr[4 * t + k] = u;
    m->nbrk[4 * t + k] = u < 0 ? -1 : ku;
    return 0;
}

/* Number of boundary faces (no neighbour). */
int64_t orc_count_boundary(const orc_mesh *m) {
    int64_t nb = 0;
    for (int64_t i = 0; i < 4 * m->nt; ++i) nb += m->nbr[i] < 0;
    return nb;
}

/* ------------------------------------------------------------------------ */
/* Ray-triangle test: Moller & Trumbore, "Fast, minimum storage ray/triangle
 * intersection", JGT 1997.  Returns 0 when the ray is parallel to the
 * triangle's plane. */
static int moller_trumbore(const double *o, const double *d, const double *v0, const double *v1,
                           const double *v2, double *t, double *b1, double *b2) {
    double e1[3], e2[3], p[3], s[3], q[3];
    sub3(v1, v0, e1); sub3(v2, v0, e2);
    cross3(d, e2, p);
    double det = dot3(e1, p);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    sub3(o, v0, s);
    *b1 = dot3(s, p) * inv;
    cross3(s, e1, q);
    *b2 = dot3(d, q) * inv;
    *t = dot3(e2, q) * inv;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* The walk.                                                                 */

typedef struct {
    const orc_mesh *m;
    int64_t n;
    const float *o, *d, *tmax;
    const int32_t *start, *entry;
    int64_t max_steps;
    int32_t *tri, *tet, *cface, *steps, *flags;
    double *t, *b1, *b2;
    int64_t lo, hi;
} walk_job;

static void walk_one(const walk_job *J, int64_t r) {
    const orc_mesh *m = J->m;
    double o[3] = {J->o[3 * r], J->o[3 * r + 1], J->o[3 * r + 2]};
    double d[3] = {J->d[3 * r], J->d[3 * r + 1], J->d[3 * r + 2]};
    double tmax = (double)J->tmax[r];
    int32_t T = J->start[r];
    int32_t kin = -1;
    int32_t flags = 0, steps = 0;
    J->tri[r] = -1; J->t[r] = INFINITY; J->b1[r] = 0; J->b2[r] = 0;
    J->cface[r] = -1; J->tet[r] = -1;
    if (J->entry[r] >= 0) {
        /* Restart through a constrained face: entry[r] = 2*c + side, the ray
         * starts in the tet on that side of triangle c and cannot cross c. */
        int32_t c = J->entry[r] >> 1, side = J->entry[r] & 1;
        T = (c < m->nc) ? m->ctet[2 * c + side] : -1;
        if (T >= 0)
            for (int k = 0; k < 4; ++k)
                if (m->fc[4 * T + k] == c) kin = k;
        if (T < 0 || kin < 0) { J->flags[r] = ORC_FLAG_BAD_START; J->steps[r] = 0; return; }
    }
    if (T < 0 || T >= m->nt) { J->flags[r] = ORC_FLAG_BAD_START; J->steps[r] = 0; return; }
    double tprev = -INFINITY;
    for (;;) {
        int best = -1;
        double tbest = INFINITY;
        for (int k = 0; k < 4; ++k) {
            if (k == kin) continue;
            const double *a = m->P + 3 * m->T[4 * T + FACE[k][0]];
            const double *b = m->P + 3 * m->T[4 * T + FACE[k][1]];
            const double *c = m->P + 3 * m->T[4 * T + FACE[k][2]];
            double ab[3], ac[3], nin[3], ao[3];
            sub3(b, a, ab); sub3(c, a, ac);
            cross3(ab, ac, nin);           /* inward normal */
            double nd = dot3(nin, d);
            if (nd < 0.0) {                /* the ray leaves through this plane */
                sub3(a, o, ao);
                double tk = dot3(nin, ao) / nd;
                if (tk < tbest) { tbest = tk; best = k; }
            }
        }
        if (best < 0) { flags |= ORC_FLAG_DEGENERATE; J->tet[r] = T; break; }
        if (tbest < tprev) flags |= ORC_FLAG_NONMONOTONE;
        else if (tbest == tprev) flags |= ORC_FLAG_TIE;
        tprev = tbest;
        J->tet[r] = T;
        if (tbest > tmax) break;                        /* ends inside T */
        int32_t c = m->fc[4 * T + best];
        if (c >= 0) {
            double th, u, v;
            const double *v0 = m->P + 3 * m->tri[3 * c], *v1 = m->P + 3 * m->tri[3 * c + 1],
                         *v2 = m->P + 3 * m->tri[3 * c + 2];
            if (moller_trumbore(o, d, v0, v1, v2, &th, &u, &v) && th <= tmax) {
                J->tri[r] = c; J->cface[r] = c; J->t[r] = th; J->b1[r] = u; J->b2[r] = v;
            }
            break;
        }
        int32_t N = m->nbr[4 * T + best];
        if (N < 0) break;                               /* mesh boundary */
        if (steps >= J->max_steps) { flags |= ORC_FLAG_STEP_LIMIT; break; }
        kin = m->nbrk[4 * T + best];
        T = N;
        ++steps;
    }
    J->steps[r] = steps;
    J->flags[r] = flags;
}

static void *walk_range(void *arg) {
    walk_job *J = (walk_job *)arg;
    for (int64_t r = J->lo; r < J->hi; ++r) walk_one(J, r);
    return NULL;
}

/* Rays: o, d float32 [n*3]; tmax float32 [n]; start = input tet id holding o
 * (used when entry < 0); entry = 2*c + side to restart through constrained
 * triangle c from the tet on its + (0) or - (1) side, else -1.  steps counts
 * the tets entered after the start tet. */
void orc_trace(const orc_mesh *m, int64_t n, const float *o, const float *d, const float *tmax,
               const int32_t *start, const int32_t *entry, int64_t max_steps, int nthreads,
               int32_t *tri, double *t, double *b1, double *b2, int32_t *tet, int32_t *cface,
               int32_t *steps, int32_t *flags) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    walk_job jobs[256];
    for (int i = 0; i < nthreads; ++i) {
        walk_job *J = &jobs[i];
        J->m = m; J->n = n; J->o = o; J->d = d; J->tmax = tmax; J->start = start; J->entry = entry;
        J->max_steps = max_steps; J->tri = tri; J->t = t; J->b1 = b1; J->b2 = b2; J->tet = tet;
        J->cface = cface; J->steps = steps; J->flags = flags;
        J->lo = n * i / nthreads; J->hi = n * (i + 1) / nthreads;
    }
    for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, walk_range, &jobs[i]);
    walk_range(&jobs[0]);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------------ */
/* Brute force: nearest constrained triangle over all of them.               */

typedef struct {
    const orc_mesh *m;
    const float *o, *d, *tmax;
    const int32_t *exclude;
    int32_t *tri;
    double *t, *b1, *b2;
    int64_t lo, hi;
} brute_job;

static void *brute_range(void *arg) {
    brute_job *J = (brute_job *)arg;
    const orc_mesh *m = J->m;
    for (int64_t r = J->lo; r < J->hi; ++r) {
        double o[3] = {J->o[3 * r], J->o[3 * r + 1], J->o[3 * r + 2]};
        double d[3] = {J->d[3 * r], J->d[3 * r + 1], J->d[3 * r + 2]};
        double tmax = (double)J->tmax[r];
        int32_t best = -1;
        double bt = INFINITY, bu = 0, bv = 0;
        for (int64_t c = 0; c < m->nc; ++c) {
            if (c == J->exclude[r]) continue;
            double th, u, v;
            const double *v0 = m->P + 3 * m->tri[3 * c], *v1 = m->P + 3 * m->tri[3 * c + 1],
                         *v2 = m->P + 3 * m->tri[3 * c + 2];
            if (!moller_trumbore(o, d, v0, v1, v2, &th, &u, &v)) continue;
            if (u < 0.0 || v < 0.0 || u + v > 1.0) continue;
            if (!(th > 0.0) || th > tmax) continue;
            if (th < bt) { bt = th; bu = u; bv = v; best = (int32_t)c; }
        }
        J->tri[r] = best; J->t[r] = bt; J->b1[r] = bu; J->b2[r] = bv;
    }
    return NULL;
}

void orc_bruteforce(const orc_mesh *m, int64_t n, const float *o, const float *d, const float *tmax,
                    const int32_t *exclude, int nthreads, int32_t *tri, double *t, double *b1,
                    double *b2) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    brute_job jobs[256];
    for (int i = 0; i < nthreads; ++i) {
        brute_job *J = &jobs[i];
        J->m = m; J->o = o; J->d = d; J->tmax = tmax; J->exclude = exclude;
        J->tri = tri; J->t = t; J->b1 = b1; J->b2 = b2;
        J->lo = n * i / nthreads; J->hi = n * (i + 1) / nthreads;
    }
    for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, brute_range, &jobs[i]);
    brute_range(&jobs[0]);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------------ */
/* Point location by brute force: the tet whose smallest barycentric
 * coordinate of q is largest (>= 0 means q is inside or on it). */

typedef struct {
    const orc_mesh *m;
    const float *q;
    int32_t *tet;
    double *minbary;
    int64_t lo, hi;
} locate_job;

static void *locate_range(void *arg) {
    locate_job *J = (locate_job *)arg;
    const orc_mesh *m = J->m;
    for (int64_t i = J->lo; i < J->hi; ++i) {
        double q[3] = {J->q[3 * i], J->q[3 * i + 1], J->q[3 * i + 2]};
        int32_t best = -1;
        double bmin = -INFINITY;
        for (int64_t t = 0; t < m->nt; ++t) {
            const int32_t *v = m->T + 4 * t;
            double vol = orient3d(m->P + 3 * v[0], m->P + 3 * v[1], m->P + 3 * v[2], m->P + 3 * v[3]);
            double mn = INFINITY;
            for (int k = 0; k < 4; ++k) {
                double w = orient3d(m->P + 3 * v[FACE[k][0]], m->P + 3 * v[FACE[k][1]],
                                    m->P + 3 * v[FACE[k][2]], q) / vol;
                if (w < mn) mn = w;
            }
            if (mn > bmin) { bmin = mn; best = (int32_t)t; }
        }
        J->tet[i] = best;
        J->minbary[i] = bmin;
    }
    return NULL;
}

void orc_locate(const orc_mesh *m, int64_t n, const float *q, int nthreads, int32_t *tet,
                double *minbary) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    locate_job jobs[256];
    for (int i = 0; i < nthreads; ++i) {
        locate_job *J = &jobs[i];
        J->m = m; J->q = q; J->tet = tet; J->minbary = minbary;
        J->lo = n * i / nthreads; J->hi = n * (i + 1) / nthreads;
    }
    for (int i = 1; i < nthreads; ++i) pthread_create(&th[i], NULL, locate_range, &jobs[i]);
    locate_range(&jobs[0]);
    for (int i = 1; i < nthreads; ++i) pthread_join(th[i], NULL);
}

/* Barycentric coordinates of q in tet t (order V0..V3). */
void orc_tet_bary(const orc_mesh *m, int32_t t, const double *q, double *w) {
    const int32_t *v = m->T + 4 * t;
    double vol = orient3d(m->P + 3 * v[0], m->P + 3 * v[1], m->P + 3 * v[2], m->P + 3 * v[3]);
    for (int k = 0; k < 4; ++k)
        w[k] = orient3d(m->P + 3 * v[FACE[k][0]], m->P + 3 * v[FACE[k][1]], m->P + 3 * v[FACE[k][2]], q) / vol;
}
