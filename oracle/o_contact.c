/* Oracle: IPC log barrier, primitive distances and the brute-force contact
 * set C(x, dhat) of Algorithm 1 (ComputeConstraintSet).  Test infrastructure
 * only.
 *
 * Readings (the paper says only that b is logarithmic, Sec. 3.1):
 *  - b(d) = -(d - dhat)^2 ln(d / dhat) for 0 < d < dhat, else 0, with d the
 *    unsigned Euclidean distance; the contact energy is kappa * b(d).
 *  - The rank-1 stiffness of Eq. 5 is k = kappa * b''(d) and n = grad d.
 *  - Pairs: point-triangle (surface vertex vs non-incident surface triangle),
 *    edge-edge (surface edges sharing no vertex; pairs whose edges are
 *    parallel to sin^2 < 1e-12 are left to the PT pairs), point-ground
 *    (surface vertex vs the plane).  Each pair is one contact; no merging of
 *    PT pairs whose closest point lies on an edge.
 *  - Distances use the full closest-point regimes; grad d comes from the
 *    closest points (the min over the primitive parameters does not depend on
 *    x, so d is differentiated at the minimiser).
 */
#include "o_internal.h"

void o_barrier(double d, double dhat, double out[3]) {
    if (!(d < dhat)) {
        out[0] = out[1] = out[2] = 0.0;
        return;
    }
    if (!(d > 0.0)) {
        out[0] = INFINITY;
        out[1] = -INFINITY;
        out[2] = INFINITY;
        return;
    }
    double q = d - dhat, L = log(d / dhat);
    out[0] = -q * q * L;
    out[1] = -2.0 * q * L - q * q / d;
    out[2] = -2.0 * L - 4.0 * q / d + q * q / (d * d);
}

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static double clamp01(double t) { return t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t); }

/* closest point of segment [a,b] to p: parameter t */
static double seg_param(const double* p, const double* a, const double* b) {
    double e[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double ee = dot3(e, e);
    if (!(ee > 0.0)) return 0.0;
    double w[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
    return clamp01(dot3(w, e) / ee);
}

static double dist_to(const double* p, const double* c) {
    double r[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
    return sqrt(dot3(r, r));
}

/* Point-triangle distance; w = barycentric weights of the closest point.
 * Interior projection if it lies in the triangle, else the best of the three
 * edge projections. */
double o_pt_distance(const double* p, const double* t0, const double* t1, const double* t2, double w[3]) {
    double e1[3] = {t1[0] - t0[0], t1[1] - t0[1], t1[2] - t0[2]};
    double e2[3] = {t2[0] - t0[0], t2[1] - t0[1], t2[2] - t0[2]};
    double r[3] = {p[0] - t0[0], p[1] - t0[1], p[2] - t0[2]};
    double a = dot3(e1, e1), b = dot3(e1, e2), c = dot3(e2, e2);
    double det = a * c - b * b;
    if (det > 1e-300 && det > 1e-14 * a * c) {
        double r1 = dot3(e1, r), r2 = dot3(e2, r);
        double u = (c * r1 - b * r2) / det;
        double v = (a * r2 - b * r1) / det;
        if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) {
            w[0] = 1.0 - u - v;
            w[1] = u;
            w[2] = v;
            double q[3];
            for (int i = 0; i < 3; ++i) q[i] = w[0] * t0[i] + w[1] * t1[i] + w[2] * t2[i];
            return dist_to(p, q);
        }
    }
    const double* T[3] = {t0, t1, t2};
    double best = INFINITY;
    for (int k = 0; k < 3; ++k) {
        const double* A = T[k];
        const double* B = T[(k + 1) % 3];
        double t = seg_param(p, A, B);
        double q[3];
        for (int i = 0; i < 3; ++i) q[i] = (1.0 - t) * A[i] + t * B[i];
        double d = dist_to(p, q);
        if (d < best) {
            best = d;
            w[0] = w[1] = w[2] = 0.0;
            w[k] = 1.0 - t;
            w[(k + 1) % 3] = t;
        }
    }
    return best;
}

/* Edge-edge distance; st = parameters on a and b.  Interior stationary point
 * if inside [0,1]^2, else the best of the four box-edge minimisers. */
double o_ee_distance(const double* a0, const double* a1, const double* b0, const double* b1, double st[2]) {
    double u[3] = {a1[0] - a0[0], a1[1] - a0[1], a1[2] - a0[2]};
    double v[3] = {b1[0] - b0[0], b1[1] - b0[1], b1[2] - b0[2]};
    double w0[3] = {a0[0] - b0[0], a0[1] - b0[1], a0[2] - b0[2]};
    double uu = dot3(u, u), uv = dot3(u, v), vv = dot3(v, v);
    double uw = dot3(u, w0), vw = dot3(v, w0);
    double det = uu * vv - uv * uv;
    if (det > 1e-300 && det > 1e-14 * uu * vv) {
        double s = (uv * vw - vv * uw) / det;
        double t = (uu * vw - uv * uw) / det;
        if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
            st[0] = s;
            st[1] = t;
            double pa[3], pb[3];
            for (int i = 0; i < 3; ++i) {
                pa[i] = a0[i] + s * u[i];
                pb[i] = b0[i] + t * v[i];
            }
            return dist_to(pa, pb);
        }
    }
    double best = INFINITY;
    double cand[4][2];
    cand[0][0] = 0.0;
    cand[0][1] = seg_param(a0, b0, b1);
    cand[1][0] = 1.0;
    cand[1][1] = seg_param(a1, b0, b1);
    cand[2][1] = 0.0;
    cand[2][0] = seg_param(b0, a0, a1);
    cand[3][1] = 1.0;
    cand[3][0] = seg_param(b1, a0, a1);
    for (int k = 0; k < 4; ++k) {
        double pa[3], pb[3];
        for (int i = 0; i < 3; ++i) {
            pa[i] = a0[i] + cand[k][0] * u[i];
            pb[i] = b0[i] + cand[k][1] * v[i];
        }
        double d = dist_to(pa, pb);
        if (d < best) {
            best = d;
            st[0] = cand[k][0];
            st[1] = cand[k][1];
        }
    }
    return best;
}

/* ---------------------------------------------------------------- list */

static void clist_push(OContactList* l, const OContact* c) {
    if (l->n == l->cap) {
        l->cap = l->cap ? 2 * l->cap : 256;
        l->c = (OContact*)realloc(l->c, sizeof(OContact) * l->cap);
    }
    l->c[l->n++] = *c;
}

void o_clist_free(OContactList* l) {
    free(l->c);
    l->c = NULL;
    l->n = l->cap = 0;
}

int o_contact_cmp(const void* a, const void* b) {
    const OContact* x = (const OContact*)a;
    const OContact* y = (const OContact*)b;
    if (x->type != y->type) return x->type < y->type ? -1 : 1;
    if (x->ida != y->ida) return x->ida < y->ida ? -1 : 1;
    if (x->idb != y->idb) return x->idb < y->idb ? -1 : 1;
    return 0;
}

static void fill_common(OScene* s, OContact* c) {
    double b[3];
    o_barrier(c->d, s->prm.dhat, b);
    c->bp = s->prm.kappa * b[1];
    c->k = s->prm.kappa * b[2];
}

/* AABB of a set of points, inflated by r */
static void box_of(const double* const* P, int n, double r, double* lo, double* hi) {
    for (int i = 0; i < 3; ++i) {
        lo[i] = INFINITY;
        hi[i] = -INFINITY;
    }
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < 3; ++i) {
            if (P[k][i] < lo[i]) lo[i] = P[k][i];
            if (P[k][i] > hi[i]) hi[i] = P[k][i];
        }
    for (int i = 0; i < 3; ++i) {
        lo[i] -= r;
        hi[i] += r;
    }
}

static int boxes_apart(const double* lo1, const double* hi1, const double* lo2, const double* hi2) {
    for (int i = 0; i < 3; ++i)
        if (hi1[i] < lo2[i] || hi2[i] < lo1[i]) return 1;
    return 0;
}

/* PT pair (surface vertex p, surface triangle f): record if d < dhat */
static void pt_check(OScene* s, const double* x, int p, int f, OContactList* out) {
    const int* T = s->sf + 3 * f;
    if (p == T[0] || p == T[1] || p == T[2]) return;
    const double* P3[3] = {x + 3 * T[0], x + 3 * T[1], x + 3 * T[2]};
    const double* xp = x + 3 * p;
    double w[3];
    double d = o_pt_distance(xp, P3[0], P3[1], P3[2], w);
    if (!(d < s->prm.dhat)) return;
    OContact c;
    memset(&c, 0, sizeof c);
    c.type = 0;
    c.v[0] = p;
    c.v[1] = T[0];
    c.v[2] = T[1];
    c.v[3] = T[2];
    c.ida = p;
    c.idb = f;
    c.d = d;
    double q[3], r[3];
    for (int k = 0; k < 3; ++k) q[k] = w[0] * P3[0][k] + w[1] * P3[1][k] + w[2] * P3[2][k];
    for (int k = 0; k < 3; ++k) r[k] = (xp[k] - q[k]) / d;
    double coef[4] = {1.0, -w[0], -w[1], -w[2]};
    for (int j = 0; j < 4; ++j)
        for (int k = 0; k < 3; ++k) c.n[3 * j + k] = coef[j] * r[k];
    fill_common(s, &c);
    clist_push(out, &c);
}

/* EE pair (surface edges i < j): record if not adjacent, not parallel, d < dhat */
static void ee_check(OScene* s, const double* x, int i, int j, OContactList* out) {
    const int* A = s->se + 2 * i;
    const int* B = s->se + 2 * j;
    if (A[0] == B[0] || A[0] == B[1] || A[1] == B[0] || A[1] == B[1]) return;
    const double* PA[2] = {x + 3 * A[0], x + 3 * A[1]};
    const double* PB[2] = {x + 3 * B[0], x + 3 * B[1]};
    double u[3], v[3], cr[3];
    for (int k = 0; k < 3; ++k) {
        u[k] = PA[1][k] - PA[0][k];
        v[k] = PB[1][k] - PB[0][k];
    }
    cr[0] = u[1] * v[2] - u[2] * v[1];
    cr[1] = u[2] * v[0] - u[0] * v[2];
    cr[2] = u[0] * v[1] - u[1] * v[0];
    if (dot3(cr, cr) < 1e-12 * dot3(u, u) * dot3(v, v)) return;
    double st[2];
    double d = o_ee_distance(PA[0], PA[1], PB[0], PB[1], st);
    if (!(d < s->prm.dhat)) return;
    OContact c;
    memset(&c, 0, sizeof c);
    c.type = 1;
    c.v[0] = A[0];
    c.v[1] = A[1];
    c.v[2] = B[0];
    c.v[3] = B[1];
    c.ida = i;
    c.idb = j;
    c.d = d;
    double r[3];
    for (int k = 0; k < 3; ++k) {
        double pa = PA[0][k] + st[0] * u[k];
        double pb = PB[0][k] + st[1] * v[k];
        r[k] = (pa - pb) / d;
    }
    double coef[4] = {1.0 - st[0], st[0], -(1.0 - st[1]), -st[1]};
    for (int jj = 0; jj < 4; ++jj)
        for (int k = 0; k < 3; ++k) c.n[3 * jj + k] = coef[jj] * r[k];
    fill_common(s, &c);
    clist_push(out, &c);
}

static void store_box(double* dst, const double* lo, const double* hi) {
    for (int r = 0; r < 3; ++r) {
        dst[r] = lo[r];
        dst[3 + r] = hi[r];
    }
}

/* Every surface PT and EE pair and every surface vertex against the ground.
 * The box test only skips pairs whose distance is provably >= dhat.  Pairs
 * come from a double loop (brute_force) or from the grid pair search over the
 * same boxes.  Output sorted by key (type, ida, idb). */
void o_find_contacts(OScene* s, const double* x, OContactList* out) {
    out->n = 0;
    double dhat = s->prm.dhat;
    double* tb = (double*)malloc(sizeof(double) * 6 * (size_t)(s->nsf + 1));
    double* pb = (double*)malloc(sizeof(double) * 6 * (size_t)(s->nsv + 1));
    double* eb = (double*)malloc(sizeof(double) * 6 * (size_t)(s->nse + 1));
    double* ebi = (double*)malloc(sizeof(double) * 6 * (size_t)(s->nse + 1));
    for (int f = 0; f < s->nsf; ++f) {
        const int* T = s->sf + 3 * f;
        const double* P3[3] = {x + 3 * T[0], x + 3 * T[1], x + 3 * T[2]};
        double lo[3], hi[3];
        box_of(P3, 3, dhat, lo, hi);
        store_box(tb + 6 * (size_t)f, lo, hi);
    }
    for (int i = 0; i < s->nsv; ++i) store_box(pb + 6 * (size_t)i, x + 3 * s->sv[i], x + 3 * s->sv[i]);
    for (int i = 0; i < s->nse; ++i) {
        const int* A = s->se + 2 * i;
        const double* PA[2] = {x + 3 * A[0], x + 3 * A[1]};
        double lo[3], hi[3];
        box_of(PA, 2, dhat, lo, hi);
        store_box(ebi + 6 * (size_t)i, lo, hi);
        box_of(PA, 2, 0.0, lo, hi);
        store_box(eb + 6 * (size_t)i, lo, hi);
    }
    if (s->prm.brute_force) {
        for (int f = 0; f < s->nsf; ++f)
            for (int i = 0; i < s->nsv; ++i) {
                const double* b = tb + 6 * (size_t)f;
                const double* xp = x + 3 * s->sv[i];
                if (xp[0] < b[0] || xp[0] > b[3] || xp[1] < b[1] || xp[1] > b[4] || xp[2] < b[2] || xp[2] > b[5])
                    continue;
                pt_check(s, x, s->sv[i], f, out);
            }
        for (int i = 0; i < s->nse; ++i)
            for (int j = i + 1; j < s->nse; ++j) {
                const double* a = ebi + 6 * (size_t)i;
                const double* b = eb + 6 * (size_t)j;
                if (boxes_apart(a, a + 3, b, b + 3)) continue;
                ee_check(s, x, i, j, out);
            }
    } else {
        double cs = s->cell > 2.0 * dhat ? s->cell : 2.0 * dhat;
        int* P = NULL;
        int np = o_box_pairs(s->nsv, pb, s->nsf, tb, 0, cs, &P);
        for (int k = 0; k < np; ++k) pt_check(s, x, s->sv[P[2 * k]], P[2 * k + 1], out);
        free(P);
        np = o_box_pairs(s->nse, ebi, s->nse, eb, 1, cs, &P);
        for (int k = 0; k < np; ++k) ee_check(s, x, P[2 * k], P[2 * k + 1], out);
        free(P);
    }
    free(tb);
    free(pb);
    free(eb);
    free(ebi);
    /* PG */
    if (s->has_ground) {
        for (int i = 0; i < s->nsv; ++i) {
            int p = s->sv[i];
            double d = dot3(s->gn, x + 3 * p) - s->goff;
            if (!(d < dhat)) continue;
            OContact c;
            memset(&c, 0, sizeof c);
            c.type = 2;
            c.v[0] = p;
            c.v[1] = c.v[2] = c.v[3] = -1;
            c.ida = p;
            c.idb = 0;
            c.d = d;
            for (int k = 0; k < 3; ++k) c.n[k] = s->gn[k];
            fill_common(s, &c);
            clist_push(out, &c);
        }
    }
    qsort(out->c, out->n, sizeof(OContact), o_contact_cmp);
}

int o_contacts(OScene* s, const double* x, int cap, int* type, int* verts, int* ids, double* dist,
               double* kstiff, double* grad12) {
    OContactList L = {0};
    o_find_contacts(s, x, &L);
    for (int i = 0; i < L.n && i < cap; ++i) {
        const OContact* c = L.c + i;
        if (type) type[i] = c->type;
        if (verts)
            for (int j = 0; j < 4; ++j) verts[4 * i + j] = c->v[j];
        if (ids) {
            ids[2 * i] = c->ida;
            ids[2 * i + 1] = c->idb;
        }
        if (dist) dist[i] = c->d;
        if (kstiff) kstiff[i] = c->k;
        if (grad12)
            for (int j = 0; j < 12; ++j) grad12[12 * i + j] = c->n[j];
    }
    int n = L.n;
    o_clist_free(&L);
    return n;
}
