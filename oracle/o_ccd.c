/* Oracle: per-subdomain conservative CCD (Sec. 4.4; supplement Sec. 3).
 * Test infrastructure only.
 *
 *  - Relative-displacement bound (supplement Eq. 29, 31):
 *      l_tight^PT = max_j |p_P - p_Tj|,  l_tight^EE = max_{i,j} |p_E1i - p_E2j|.
 *  - Lower bound alpha_l = d_min / l_tight.  Reading: d_min = (1 - s) d0 with
 *    s = ccd_shrink and d0 the pair's current distance.
 *  - Coplanarity cubic f(t) = det[x1 - x0, x2 - x0, x3 - x0](t) with
 *    x_i(t) = x_i + t p_i; PT uses (t0, t1, t2, p), EE uses (a0, a1, b0, b1).
 *  - Safe step by cubic analysis (supplement Algorithm 2) and the fixed
 *    16-step bisection (supplement Algorithm 1).  Readings of the garbled
 *    pseudo-code: the bisection's same-sign branch moves the safe end (its
 *    value keeps the same sign, so updating it or not is equivalent); every
 *    monotone segment boundary e in (x, 1] is tested in order; on a sign
 *    change the step is x itself if x has moved past its start
 *    max(0, alpha_l) (same as x > alpha_l for alpha_l >= 0), else the
 *    bisection of [x, e]; with no sign change the step is 1.  sign(0) is its
 *    own value.
 *  - Candidates: PT / EE pairs whose swept boxes over [x, x + p] overlap,
 *    found by brute force over all pairs; point-ground pairs take
 *    alpha = min(1, (1 - s) d0 / (-n . p)) when moving toward the plane.
 *  - alpha_d = min(1, min over candidate pairs with a vertex in d).
 *  - Reading for pairs straddling subdomains (the paper is silent): the
 *    actual motion q_v = alpha_d(v) p_v is re-checked with the same cubic
 *    analysis on t in [0, 1]; every subdomain touched by a pair whose safe
 *    fraction rho < 1 takes the smallest alpha among that pair's subdomains
 *    (the pair then moves uniformly along a segment already checked).  A
 *    pass sees the alphas of the previous pass.  At most O_CCD_PASSES
 *    passes; if the last still finds a violation, every subdomain takes the
 *    uniform step min_d alpha_d, which is safe by construction.  Neither
 *    outcome is ever below that uniform step.
 */
#include "o_internal.h"

#define O_CCD_PASSES 8

static double sgn(double v) { return (v > 0.0) - (v < 0.0); }

static double cubic_eval(const double c[4], double t) { return ((c[3] * t + c[2]) * t + c[1]) * t + c[0]; }

double o_safe_bisect(const double coef[4], double xs, double xu, double ys, double yu) {
    (void)yu;
    for (int i = 0; i < 16; ++i) {
        double xm = 0.5 * (xs + xu);
        double ym = cubic_eval(coef, xm);
        if (sgn(ys) != sgn(ym)) {
            xu = xm;
        } else {
            xs = xm;
            ys = ym;
        }
    }
    return xs;
}

double o_cubic_safe(const double coef[4], double alpha_l) {
    if (alpha_l >= 1.0) return 1.0;
    double a = coef[3], b = coef[2], c = coef[1];
    double x = alpha_l > 0.0 ? alpha_l : 0.0;
    const double x_start = x;
    double y = cubic_eval(coef, x);
    if (y == 0.0) return x;
    /* monotone segment boundaries in (x, 1): critical points of f */
    double ends[3];
    int ne = 0;
    double disc = b * b - 3.0 * a * c;
    if (disc > 0.0) {
        double q = -(b + (b >= 0.0 ? 1.0 : -1.0) * sqrt(disc));
        double r1 = q / (3.0 * a), r2 = c / q;
        double lo = r1 < r2 ? r1 : r2, hi = r1 < r2 ? r2 : r1;
        if (lo > x && lo < 1.0) ends[ne++] = lo;
        if (hi > x && hi < 1.0 && hi > lo) ends[ne++] = hi;
    } else if (disc == 0.0 && a != 0.0) {
        double ti = -b / (3.0 * a);
        if (ti > x && ti < 1.0) ends[ne++] = ti;
    }
    ends[ne++] = 1.0;
    for (int k = 0; k < ne; ++k) {
        double e = ends[k];
        double ye = cubic_eval(coef, e);
        if (sgn(y) != sgn(ye)) {
            if (x > x_start) return x;
            return o_safe_bisect(coef, x, e, y, ye);
        }
        x = e;
        y = ye;
    }
    return 1.0;
}

/* det[a + t da, b + t db, c + t dc] = sum_k coef[k] t^k */
static void det_cubic(const double* A, const double* dA, const double* B, const double* dB, const double* C,
                      const double* dC, double coef[4]) {
#define CROSS(u, v, o) \
    o[0] = u[1] * v[2] - u[2] * v[1]; \
    o[1] = u[2] * v[0] - u[0] * v[2]; \
    o[2] = u[0] * v[1] - u[1] * v[0];
#define DOT(u, v) (u[0] * v[0] + u[1] * v[1] + u[2] * v[2])
    double bc[3], bdc[3], dbc[3], dbdc[3];
    CROSS(B, C, bc);
    CROSS(B, dC, bdc);
    CROSS(dB, C, dbc);
    CROSS(dB, dC, dbdc);
    coef[0] = DOT(A, bc);
    coef[1] = DOT(dA, bc) + DOT(A, dbc) + DOT(A, bdc);
    coef[2] = DOT(dA, dbc) + DOT(dA, bdc) + DOT(A, dbdc);
    coef[3] = DOT(dA, dbdc);
#undef CROSS
#undef DOT
}

/* x4, p4: 4 points (12 doubles) in the order (t0, t1, t2, p) for PT */
void o_pt_cubic(const double* x4, const double* p4, double coef[4]) {
    double A[3], dA[3], B[3], dB[3], C[3], dC[3];
    for (int i = 0; i < 3; ++i) {
        A[i] = x4[3 + i] - x4[i];
        dA[i] = p4[3 + i] - p4[i];
        B[i] = x4[6 + i] - x4[i];
        dB[i] = p4[6 + i] - p4[i];
        C[i] = x4[9 + i] - x4[i];
        dC[i] = p4[9 + i] - p4[i];
    }
    det_cubic(A, dA, B, dB, C, dC, coef);
}

/* order (a0, a1, b0, b1): det[b0 - a0, a1 - a0, b1 - a0] */
void o_ee_cubic(const double* x4, const double* p4, double coef[4]) {
    double A[3], dA[3], B[3], dB[3], C[3], dC[3];
    for (int i = 0; i < 3; ++i) {
        A[i] = x4[6 + i] - x4[i];
        dA[i] = p4[6 + i] - p4[i];
        B[i] = x4[3 + i] - x4[i];
        dB[i] = p4[3 + i] - p4[i];
        C[i] = x4[9 + i] - x4[i];
        dC[i] = p4[9 + i] - p4[i];
    }
    det_cubic(A, dA, B, dB, C, dC, coef);
}

static double norm_diff(const double* a, const double* b) {
    double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
    return sqrt(d0 * d0 + d1 * d1 + d2 * d2);
}

/* p4 order (p, t0, t1, t2) */
double o_ltight_pt(const double* p4) {
    double l = 0.0;
    for (int j = 1; j < 4; ++j) {
        double d = norm_diff(p4, p4 + 3 * j);
        if (d > l) l = d;
    }
    return l;
}

/* p4 order (a0, a1, b0, b1) */
double o_ltight_ee(const double* p4) {
    double l = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int j = 2; j < 4; ++j) {
            double d = norm_diff(p4 + 3 * i, p4 + 3 * j);
            if (d > l) l = d;
        }
    return l;
}

/* supplement Eq. 23: max |p_P| + max_j |p_Tj|, p4 order (p, t0, t1, t2) */
double o_loriginal_pt(const double* p4) {
    double z[3] = {0, 0, 0};
    double a = norm_diff(p4, z), b = 0.0;
    for (int j = 1; j < 4; ++j) {
        double d = norm_diff(p4 + 3 * j, z);
        if (d > b) b = d;
    }
    return a + b;
}

/* distance of the pair at X + t Q (PT: p, t0, t1, t2; EE: a0, a1, b0, b1) */
static double dist_at(int kind, const double* X, const double* Q, double t) {
    double Y[12], w[3], st[2];
    for (int i = 0; i < 12; ++i) Y[i] = X[i] + t * Q[i];
    return kind == 0 ? o_pt_distance(Y, Y + 3, Y + 6, Y + 9, w) : o_ee_distance(Y, Y + 3, Y + 6, Y + 9, st);
}

/* safe fraction of the motion x + t q, t in [0,1], for a PT (kind 0) or
 * EE (kind 1) pair on vertices v[4] (PT: p, t0, t1, t2). */
/* safe fraction of the motion X + t Q, t in [0,1], of one PT (kind 0:
 * p, t0, t1, t2) or EE (kind 1: a0, a1, b0, b1) pair given as 4 x 3
 * positions and displacements. */
double o_pair_safe(int kind, const double* X, const double* Q, double shrink, double dhat) {
    double d0, l, coef[4];
    if (kind == 0) {
        double w[3];
        d0 = o_pt_distance(X, X + 3, X + 6, X + 9, w);
        l = o_ltight_pt(Q);
        /* cubic wants (t0, t1, t2, p) */
        double X2[12], Q2[12];
        memcpy(X2, X + 3, sizeof(double) * 9);
        memcpy(X2 + 9, X, sizeof(double) * 3);
        memcpy(Q2, Q + 3, sizeof(double) * 9);
        memcpy(Q2 + 9, Q, sizeof(double) * 3);
        o_pt_cubic(X2, Q2, coef);
    } else {
        double st[2];
        d0 = o_ee_distance(X, X + 3, X + 6, X + 9, st);
        l = o_ltight_ee(Q);
        o_ee_cubic(X, Q, coef);
    }
    double al = l > 0.0 ? (1.0 - shrink) * d0 / l : INFINITY;
    double a = o_cubic_safe(coef, al);
    /* The coplanarity walk only rules out crossing: a grazing motion may end
     * arbitrarily close to contact.  Reading: when the end of the step lies
     * closer than s * min(d0, dhat), the step is cut back by bisection between
     * the conservative bound alpha_l (where d >= s d0 holds) and the walk's
     * result, 12 halvings. */
    if (a > al) {
        double thr = shrink * (d0 < dhat ? d0 : dhat);
        if (dist_at(kind, X, Q, a) < thr) {
            double lo = al > 0.0 ? al : 0.0, hi = a;
            for (int it = 0; it < 12; ++it) {
                double mid = 0.5 * (lo + hi);
                if (dist_at(kind, X, Q, mid) >= thr)
                    lo = mid;
                else
                    hi = mid;
            }
            a = lo;
        }
    }
    return a;
}

static double pair_safe(const OScene* s, int kind, const int* v, const double* x, const double* q) {
    double X[12], Q[12];
    for (int j = 0; j < 4; ++j)
        for (int r = 0; r < 3; ++r) {
            X[3 * j + r] = x[3 * v[j] + r];
            Q[3 * j + r] = q[3 * v[j] + r];
        }
    return o_pair_safe(kind, X, Q, s->prm.ccd_shrink, s->prm.dhat);
}

static void swept_box(const double* x, const double* p, const int* v, int n, double* lo, double* hi) {
    for (int i = 0; i < 3; ++i) {
        lo[i] = INFINITY;
        hi[i] = -INFINITY;
    }
    for (int k = 0; k < n; ++k)
        for (int i = 0; i < 3; ++i) {
            double a = x[3 * v[k] + i], b = a + p[3 * v[k] + i];
            double mn = a < b ? a : b, mx = a < b ? b : a;
            if (mn < lo[i]) lo[i] = mn;
            if (mx > hi[i]) hi[i] = mx;
        }
}

static int overlap(const double* lo1, const double* hi1, const double* lo2, const double* hi2) {
    for (int i = 0; i < 3; ++i)
        if (hi1[i] < lo2[i] || hi2[i] < lo1[i]) return 0;
    return 1;
}

typedef struct Cand {
    int kind;  /* 0 PT, 1 EE */
    int v[4];
} Cand;

/* Step sizes for one grouping of the vertices (level-0 subdomains or bodies):
 * alpha_g = min(1, min over candidate pairs and point-ground pairs touching
 * g), then verification of the pairs straddling groups with the actual motion
 * alpha_g(v) p_v.  Returns the number of passes, -1 for the uniform fallback. */
static int group_steps(OScene* s, const double* x, const double* p, const Cand* cand, int nc, const double* apair,
                       const double* apg, const int* grp, int ng, double* alpha) {
    for (int g = 0; g < ng; ++g) alpha[g] = 1.0;
    for (int k = 0; k < nc; ++k)
        for (int j = 0; j < 4; ++j) {
            int g = grp[cand[k].v[j]];
            if (apair[k] < alpha[g]) alpha[g] = apair[k];
        }
    for (int i = 0; i < s->nsv; ++i) {
        int g = grp[s->sv[i]];
        if (apg[i] < alpha[g]) alpha[g] = apg[i];
    }
    double* q = (double*)malloc(sizeof(double) * 3 * (size_t)s->nv);
    double* shrink = (double*)malloc(sizeof(double) * ng);
    double amin = 1.0;
    for (int g = 0; g < ng; ++g)
        if (alpha[g] < amin) amin = alpha[g];
    int passes = 0, ok = 0;
    for (int pass = 0; pass < O_CCD_PASSES; ++pass) {
        ++passes;
        for (int v = 0; v < s->nv; ++v)
            for (int r = 0; r < 3; ++r) q[3 * v + r] = alpha[grp[v]] * p[3 * v + r];
        for (int g = 0; g < ng; ++g) shrink[g] = alpha[g];
        int viol = 0;
        for (int k = 0; k < nc; ++k) {
            const int* v = cand[k].v;
            int g0 = grp[v[0]];
            if (grp[v[1]] == g0 && grp[v[2]] == g0 && grp[v[3]] == g0) continue;
            double rho = pair_safe(s, cand[k].kind, v, x, q);
            if (rho < 1.0) {
                /* equalise: every group of the pair takes the pair's smallest
                 * alpha, so the pair moves uniformly */
                viol = 1;
                double m = alpha[grp[v[0]]];
                for (int j = 1; j < 4; ++j)
                    if (alpha[grp[v[j]]] < m) m = alpha[grp[v[j]]];
                for (int j = 0; j < 4; ++j)
                    if (m < shrink[grp[v[j]]]) shrink[grp[v[j]]] = m;
            }
        }
        if (!viol) {
            ok = 1;
            break;
        }
        for (int g = 0; g < ng; ++g) alpha[g] = shrink[g];
    }
    if (!ok) {
        for (int g = 0; g < ng; ++g) alpha[g] = amin;
        passes = -1;
    }
    free(q);
    free(shrink);
    return passes;
}

int o_ccd(OScene* s, const double* x, const double* p, double* alpha, double* alpha_body, int* passes_body) {
    Cand* cand = NULL;
    int nc = 0, cc = 0;
    /* swept boxes of surface points, triangles and edges over [x, x + p] */
    double* pb = (double*)malloc(sizeof(double) * 6 * (size_t)(s->nsv + 1));
    double* tb = (double*)malloc(sizeof(double) * 6 * (size_t)(s->nsf + 1));
    double* eb = (double*)malloc(sizeof(double) * 6 * (size_t)(s->nse + 1));
    double pmax = 0.0;
    for (int i = 0; i < s->nsv; ++i) {
        swept_box(x, p, s->sv + i, 1, pb + 6 * (size_t)i, pb + 6 * (size_t)i + 3);
        const double* pv = p + 3 * s->sv[i];
        double l = sqrt(pv[0] * pv[0] + pv[1] * pv[1] + pv[2] * pv[2]);
        if (l > pmax) pmax = l;
    }
    for (int f = 0; f < s->nsf; ++f) swept_box(x, p, s->sf + 3 * f, 3, tb + 6 * (size_t)f, tb + 6 * (size_t)f + 3);
    for (int i = 0; i < s->nse; ++i) swept_box(x, p, s->se + 2 * i, 2, eb + 6 * (size_t)i, eb + 6 * (size_t)i + 3);
    int *PT = NULL, *EE = NULL, npt = 0, nee = 0;
    if (s->prm.brute_force) {
        int cap = 0;
        for (int i = 0; i < s->nsv; ++i)
            for (int f = 0; f < s->nsf; ++f) {
                const double* a = pb + 6 * (size_t)i;
                const double* b = tb + 6 * (size_t)f;
                if (!overlap(a, a + 3, b, b + 3)) continue;
                if (npt == cap) {
                    cap = cap ? 2 * cap : 1024;
                    PT = (int*)realloc(PT, sizeof(int) * 2 * cap);
                }
                PT[2 * npt] = i;
                PT[2 * npt + 1] = f;
                ++npt;
            }
        cap = 0;
        for (int i = 0; i < s->nse; ++i)
            for (int j = i + 1; j < s->nse; ++j) {
                const double* a = eb + 6 * (size_t)i;
                const double* b = eb + 6 * (size_t)j;
                if (!overlap(a, a + 3, b, b + 3)) continue;
                if (nee == cap) {
                    cap = cap ? 2 * cap : 1024;
                    EE = (int*)realloc(EE, sizeof(int) * 2 * cap);
                }
                EE[2 * nee] = i;
                EE[2 * nee + 1] = j;
                ++nee;
            }
    } else {
        double cs = s->cell > pmax ? s->cell : pmax;
        npt = o_box_pairs(s->nsv, pb, s->nsf, tb, 0, cs, &PT);
        nee = o_box_pairs(s->nse, eb, s->nse, eb, 1, cs, &EE);
    }
    for (int k = 0; k < npt; ++k) {
        int pv = s->sv[PT[2 * k]];
        const int* T = s->sf + 3 * PT[2 * k + 1];
        if (pv == T[0] || pv == T[1] || pv == T[2]) continue;
        if (nc == cc) {
            cc = cc ? 2 * cc : 1024;
            cand = (Cand*)realloc(cand, sizeof(Cand) * cc);
        }
        Cand* c = cand + nc++;
        c->kind = 0;
        c->v[0] = pv;
        c->v[1] = T[0];
        c->v[2] = T[1];
        c->v[3] = T[2];
    }
    for (int k = 0; k < nee; ++k) {
        const int* A = s->se + 2 * EE[2 * k];
        const int* B = s->se + 2 * EE[2 * k + 1];
        if (A[0] == B[0] || A[0] == B[1] || A[1] == B[0] || A[1] == B[1]) continue;
        if (nc == cc) {
            cc = cc ? 2 * cc : 1024;
            cand = (Cand*)realloc(cand, sizeof(Cand) * cc);
        }
        Cand* c = cand + nc++;
        c->kind = 1;
        c->v[0] = A[0];
        c->v[1] = A[1];
        c->v[2] = B[0];
        c->v[3] = B[1];
    }
    free(PT);
    free(EE);
    free(pb);
    free(tb);
    free(eb);
    /* per-pair steps, computed once for both groupings */
    double* apair = (double*)malloc(sizeof(double) * (nc + 1));
    for (int k = 0; k < nc; ++k) apair[k] = pair_safe(s, cand[k].kind, cand[k].v, x, p);
    double* apg = (double*)malloc(sizeof(double) * (s->nsv + 1));
    for (int i = 0; i < s->nsv; ++i) {
        int v = s->sv[i];
        apg[i] = 1.0;
        if (!s->has_ground) continue;
        double vn = s->gn[0] * p[3 * v] + s->gn[1] * p[3 * v + 1] + s->gn[2] * p[3 * v + 2];
        if (!(vn < 0.0)) continue;
        double d0 = s->gn[0] * x[3 * v] + s->gn[1] * x[3 * v + 1] + s->gn[2] * x[3 * v + 2] - s->goff;
        double a = (1.0 - s->prm.ccd_shrink) * d0 / (-vn);
        if (a > 1.0) a = 1.0;
        if (!(a > 0.0)) a = 0.0;
        apg[i] = a;
    }
    int passes = group_steps(s, x, p, cand, nc, apair, apg, s->group_of[0], s->ngroups[0], alpha);
    if (alpha_body) {
        int pb2 = group_steps(s, x, p, cand, nc, apair, apg, s->body, s->nbody, alpha_body);
        if (passes_body) *passes_body = pb2;
    }
    free(apair);
    free(apg);
    free(cand);
    return passes;
}
