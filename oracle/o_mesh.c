/* Oracle: scene set-up, surface extraction, lumped mass, rest shape and the
 * MAS subdomain hierarchy.  Test infrastructure only.
 *
 * Readings (the paper is silent):
 *  - Lumped mass: rho * V / 4 to each tet vertex.
 *  - Lame parameters from (E, nu): mu = E / (2 (1 + nu)),
 *    lambda = E nu / ((1 + nu)(1 - 2 nu)).
 *  - Surface = tet faces that occur once; surface edges = edges of surface
 *    triangles; both in lexicographic order of their sorted vertex ids.
 *  - Hierarchy (supplement Sec. 1.2): level-0 nodes are vertices; a greedy
 *    BFS over mesh adjacency (start at the lowest unvisited node, neighbours
 *    in ascending id) orders the nodes, and consecutive runs of `subdomain`
 *    nodes form the subdomains.  Level l+1 nodes are level-l subdomains, two
 *    being adjacent when a mesh edge joins them.  A level with at most
 *    `subdomain` nodes is one subdomain and is the last; at most levels_max
 *    levels.
 */
#include "o_internal.h"
#include <stdarg.h>

static char g_err[512];

void o_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

const char* o_last_error(void) { return g_err; }

/* ---------------------------------------------------------------- dense */

/* Cholesky A = L L^T in place (lower): the plain column algorithm.
 * Reading for numerically singular SPD blocks (stiff rank-1 contact terms,
 * the block inverse of supplement Sec. 1.1): a pivot (Schur-complement
 * diagonal) at or below 1e-12 of the original diagonal entry is floored
 * there, i.e. A plus a tiny non-negative diagonal shift is factorised.  An
 * SPD block whose exact pivots all exceed that floor is factorised without
 * change.  Every floored pivot is counted (o_chol_floors), so that tests can
 * check that no parity state reaches the floor.  Returns the number of
 * floored pivots of this call. */
static long long g_chol_floors = 0;

#ifdef _OPENMP
#include <omp.h>
#endif

/* Host threads for the loops whose iterations are independent (per-tet
 * Hessians, per-subdomain factorisations); results do not depend on it. */
int o_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

long long o_chol_floors(int reset) {
    long long n = g_chol_floors;
    if (reset) g_chol_floors = 0;
    return n;
}

int o_chol(int n, double* A) {
    int floored = 0;
    for (int j = 0; j < n; ++j) {
        double a0 = A[j * n + j];
        double s = a0;
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        double fl = 1e-12 * a0;
        if (!(s > fl)) {
            s = fl > 0.0 ? fl : 1.0;
            ++floored;
        }
        double l = sqrt(s);
        A[j * n + j] = l;
        for (int i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / l;
        }
        for (int i = 0; i < j; ++i) A[i * n + j] = 0.0;
    }
    if (floored) {
#pragma omp atomic
        g_chol_floors += floored;
    }
    return floored;
}

/* Dense SPD inverse through o_chol (test access to the factorisation):
 * out = A^-1 column by column; returns the floored pivots. */
int o_chol_inverse(int n, const double* A, double* out) {
    double* L = (double*)malloc(sizeof(double) * n * n);
    double* e = (double*)malloc(sizeof(double) * n);
    memcpy(L, A, sizeof(double) * n * n);
    int f = o_chol(n, L);
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) e[i] = i == c ? 1.0 : 0.0;
        o_chol_solve(n, L, e);
        for (int i = 0; i < n; ++i) out[i * n + c] = e[i];
    }
    free(L);
    free(e);
    return f;
}

void o_chol_solve(int n, const double* L, double* b) {
    for (int i = 0; i < n; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= L[i * n + k] * b[k];
        b[i] = t / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = b[i];
        for (int k = i + 1; k < n; ++k) t -= L[k * n + i] * b[k];
        b[i] = t / L[i * n + i];
    }
}

/* Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix.  A is
 * destroyed; Q holds eigenvectors as columns. */
void o_jacobi_eig(int n, double* A, double* evals, double* Q) {
    for (int i = 0; i < n * n; ++i) Q[i] = 0.0;
    for (int i = 0; i < n; ++i) Q[i * n + i] = 1.0;
    double total = 0.0;
    for (int i = 0; i < n * n; ++i) total += A[i] * A[i];
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) off += A[i * n + j] * A[i * n + j];
        if (off <= 1e-32 * total || off == 0.0) break;
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double apq = A[p * n + q];
                if (apq == 0.0) continue;
                double app = A[p * n + p], aqq = A[q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < n; ++k) {
                    double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - sn * akq;
                    A[k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - sn * aqk;
                    A[q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double qkp = Q[k * n + p], qkq = Q[k * n + q];
                    Q[k * n + p] = c * qkp - sn * qkq;
                    Q[k * n + q] = sn * qkp + c * qkq;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) evals[i] = A[i * n + i];
}

/* Replace a symmetric matrix by its PSD projection: negative eigenvalues
 * clamped to zero (the projection used for the elastic Hessian). */
void o_psd_project(int n, double* A) {
    double* W = (double*)malloc(sizeof(double) * n * n);
    double* Q = (double*)malloc(sizeof(double) * n * n);
    double* e = (double*)malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) W[i * n + j] = 0.5 * (A[i * n + j] + A[j * n + i]);
    o_jacobi_eig(n, W, e, Q);
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k)
                if (e[k] > 0.0) s += Q[i * n + k] * e[k] * Q[j * n + k];
            A[i * n + j] = s;
        }
    }
    free(W);
    free(Q);
    free(e);
}

/* ---------------------------------------------------------------- mesh */

static int cmp_int3(const void* a, const void* b) {
    const int* x = (const int*)a;
    const int* y = (const int*)b;
    for (int i = 0; i < 3; ++i)
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

static int cmp_int2(const void* a, const void* b) {
    const int* x = (const int*)a;
    const int* y = (const int*)b;
    for (int i = 0; i < 2; ++i)
        if (x[i] != y[i]) return x[i] < y[i] ? -1 : 1;
    return 0;
}

static int cmp_int(const void* a, const void* b) {
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

static void sort3(int* a) {
    int t;
    if (a[0] > a[1]) { t = a[0]; a[0] = a[1]; a[1] = t; }
    if (a[1] > a[2]) { t = a[1]; a[1] = a[2]; a[2] = t; }
    if (a[0] > a[1]) { t = a[0]; a[0] = a[1]; a[1] = t; }
}

int o_build_mesh(OScene* s) {
    int nt = s->nt, nv = s->nv;
    /* rest shape, volume, Lame, mass */
    s->mu = (double*)calloc(nt, sizeof(double));
    s->lam = (double*)calloc(nt, sizeof(double));
    s->vol = (double*)calloc(nt, sizeof(double));
    s->Dm_inv = (double*)calloc(9 * (size_t)nt, sizeof(double));
    s->mass = (double*)calloc(nv, sizeof(double));
    for (int t = 0; t < nt; ++t) {
        const int* q = s->tets + 4 * t;
        double Dm[9];
        for (int j = 0; j < 3; ++j)
            for (int r = 0; r < 3; ++r)
                Dm[r * 3 + j] = s->x_rest[3 * q[j + 1] + r] - s->x_rest[3 * q[0] + r];
        double det = Dm[0] * (Dm[4] * Dm[8] - Dm[5] * Dm[7]) - Dm[1] * (Dm[3] * Dm[8] - Dm[5] * Dm[6]) +
                     Dm[2] * (Dm[3] * Dm[7] - Dm[4] * Dm[6]);
        if (!(det > 0.0)) {
            o_set_error("tet %d has non-positive rest volume", t);
            return -1;
        }
        double* B = s->Dm_inv + 9 * t;
        B[0] = (Dm[4] * Dm[8] - Dm[5] * Dm[7]) / det;
        B[1] = (Dm[2] * Dm[7] - Dm[1] * Dm[8]) / det;
        B[2] = (Dm[1] * Dm[5] - Dm[2] * Dm[4]) / det;
        B[3] = (Dm[5] * Dm[6] - Dm[3] * Dm[8]) / det;
        B[4] = (Dm[0] * Dm[8] - Dm[2] * Dm[6]) / det;
        B[5] = (Dm[2] * Dm[3] - Dm[0] * Dm[5]) / det;
        B[6] = (Dm[3] * Dm[7] - Dm[4] * Dm[6]) / det;
        B[7] = (Dm[1] * Dm[6] - Dm[0] * Dm[7]) / det;
        B[8] = (Dm[0] * Dm[4] - Dm[1] * Dm[3]) / det;
        s->vol[t] = det / 6.0;
    }
    return 0;
}

/* ---------------------------------------------------------------- surface */

static int build_surface(OScene* s) {
    int nt = s->nt;
    int* faces = (int*)malloc(sizeof(int) * 6 * 4 * (size_t)nt); /* sorted(3) + oriented(3) */
    static const int fidx[4][3] = {{0, 2, 1}, {0, 1, 3}, {0, 3, 2}, {1, 2, 3}};
    for (int t = 0; t < nt; ++t) {
        const int* q = s->tets + 4 * t;
        for (int f = 0; f < 4; ++f) {
            int* r = faces + 6 * (4 * t + f);
            for (int j = 0; j < 3; ++j) r[3 + j] = q[fidx[f][j]];
            r[0] = r[3]; r[1] = r[4]; r[2] = r[5];
            sort3(r);
        }
    }
    /* sort 6-int records by the sorted triple */
    qsort(faces, 4 * (size_t)nt, sizeof(int) * 6, cmp_int3);
    int nf = 4 * nt, nsf = 0;
    int* sf = (int*)malloc(sizeof(int) * 3 * (size_t)nf);
    for (int i = 0; i < nf;) {
        int j = i + 1;
        while (j < nf && cmp_int3(faces + 6 * i, faces + 6 * j) == 0) ++j;
        if (j - i == 1) {
            memcpy(sf + 3 * nsf, faces + 6 * i + 3, sizeof(int) * 3);
            ++nsf;
        }
        i = j;
    }
    free(faces);
    s->nsf = nsf;
    s->sf = sf;
    /* edges */
    int* e = (int*)malloc(sizeof(int) * 2 * 3 * (size_t)(nsf + 1));
    for (int f = 0; f < nsf; ++f) {
        for (int j = 0; j < 3; ++j) {
            int a = sf[3 * f + j], b = sf[3 * f + (j + 1) % 3];
            e[2 * (3 * f + j)] = a < b ? a : b;
            e[2 * (3 * f + j) + 1] = a < b ? b : a;
        }
    }
    qsort(e, 3 * (size_t)nsf, sizeof(int) * 2, cmp_int2);
    int nse = 0;
    for (int i = 0; i < 3 * nsf; ++i) {
        if (nse > 0 && e[2 * (nse - 1)] == e[2 * i] && e[2 * (nse - 1) + 1] == e[2 * i + 1]) continue;
        e[2 * nse] = e[2 * i];
        e[2 * nse + 1] = e[2 * i + 1];
        ++nse;
    }
    s->nse = nse;
    s->se = e;
    double len = 0.0;
    for (int i = 0; i < nse; ++i) {
        double d2 = 0.0;
        for (int r = 0; r < 3; ++r) {
            double d = s->x_rest[3 * e[2 * i] + r] - s->x_rest[3 * e[2 * i + 1] + r];
            d2 += d * d;
        }
        len += sqrt(d2);
    }
    s->cell = nse > 0 ? len / nse : 1.0;
    /* vertices */
    s->on_surface = (int*)calloc(s->nv, sizeof(int));
    for (int i = 0; i < 3 * nsf; ++i) s->on_surface[sf[i]] = 1;
    s->nsv = 0;
    for (int v = 0; v < s->nv; ++v) s->nsv += s->on_surface[v];
    s->sv = (int*)malloc(sizeof(int) * (s->nsv + 1));
    int k = 0;
    for (int v = 0; v < s->nv; ++v)
        if (s->on_surface[v]) s->sv[k++] = v;
    return 0;
}

static void build_adjacency(OScene* s) {
    int nt = s->nt, nv = s->nv;
    int* pairs = (int*)malloc(sizeof(int) * 2 * 12 * (size_t)nt);
    int np = 0;
    for (int t = 0; t < nt; ++t) {
        const int* q = s->tets + 4 * t;
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b)
                if (a != b) {
                    pairs[2 * np] = q[a];
                    pairs[2 * np + 1] = q[b];
                    ++np;
                }
    }
    qsort(pairs, np, sizeof(int) * 2, cmp_int2);
    s->adj_ptr = (int*)calloc(nv + 1, sizeof(int));
    s->adj = (int*)malloc(sizeof(int) * (np + 1));
    int na = 0;
    for (int i = 0; i < np; ++i) {
        if (i > 0 && pairs[2 * i] == pairs[2 * i - 2] && pairs[2 * i + 1] == pairs[2 * i - 1]) continue;
        s->adj[na++] = pairs[2 * i + 1];
        s->adj_ptr[pairs[2 * i] + 1]++;
    }
    for (int v = 0; v < nv; ++v) s->adj_ptr[v + 1] += s->adj_ptr[v];
    free(pairs);
}

/* BFS ordering of a graph given as CSR with ascending neighbour lists. */
static void bfs_order(int n, const int* ptr, const int* nb, int* order) {
    char* seen = (char*)calloc(n, 1);
    int head = 0, tail = 0;
    for (int start = 0; start < n; ++start) {
        if (seen[start]) continue;
        seen[start] = 1;
        order[tail++] = start;
        while (head < tail) {
            int u = order[head++];
            for (int k = ptr[u]; k < ptr[u + 1]; ++k) {
                int w = nb[k];
                if (!seen[w]) {
                    seen[w] = 1;
                    order[tail++] = w;
                }
            }
        }
    }
    free(seen);
}

/* bodies: connected components over tet edges, numbered in order of their
 * lowest vertex id */
static void build_bodies(OScene* s) {
    s->body = (int*)malloc(sizeof(int) * s->nv);
    for (int v = 0; v < s->nv; ++v) s->body[v] = -1;
    int* stack = (int*)malloc(sizeof(int) * s->nv);
    s->nbody = 0;
    for (int v0 = 0; v0 < s->nv; ++v0) {
        if (s->body[v0] >= 0) continue;
        int top = 0;
        stack[top++] = v0;
        s->body[v0] = s->nbody;
        while (top > 0) {
            int u = stack[--top];
            for (int k = s->adj_ptr[u]; k < s->adj_ptr[u + 1]; ++k) {
                int w = s->adj[k];
                if (s->body[w] < 0) {
                    s->body[w] = s->nbody;
                    stack[top++] = w;
                }
            }
        }
        s->nbody++;
    }
    free(stack);
}

int o_build_hierarchy(OScene* s) {
    int S = s->prm.subdomain;
    int n = s->nv;
    /* level-0 graph = vertex adjacency */
    int* ptr = (int*)malloc(sizeof(int) * (n + 1));
    memcpy(ptr, s->adj_ptr, sizeof(int) * (n + 1));
    int* nb = (int*)malloc(sizeof(int) * (ptr[n] + 1));
    memcpy(nb, s->adj, sizeof(int) * ptr[n]);
    s->nlev = 0;
    for (int l = 0; l < s->prm.levels_max && l < O_MAX_LEVELS; ++l) {
        s->nnodes[l] = n;
        int* order = (int*)malloc(sizeof(int) * n);
        int last = (n <= S) || (l == s->prm.levels_max - 1) || (l == O_MAX_LEVELS - 1);
        if (n <= S) {
            for (int i = 0; i < n; ++i) order[i] = i;
        } else {
            bfs_order(n, ptr, nb, order);
        }
        int ng = (n + S - 1) / S;
        s->ngroups[l] = ng;
        s->group_of[l] = (int*)malloc(sizeof(int) * n);
        s->slot_of[l] = (int*)malloc(sizeof(int) * n);
        s->gsize[l] = (int*)calloc(ng, sizeof(int));
        for (int i = 0; i < n; ++i) {
            s->group_of[l][order[i]] = i / S;
            s->slot_of[l][order[i]] = i % S;
            s->gsize[l][i / S]++;
        }
        s->members[l] = order;
        s->node_of_vert[l] = (int*)malloc(sizeof(int) * s->nv);
        if (l == 0) {
            for (int v = 0; v < s->nv; ++v) s->node_of_vert[0][v] = v;
        } else {
            for (int v = 0; v < s->nv; ++v)
                s->node_of_vert[l][v] = s->group_of[l - 1][s->node_of_vert[l - 1][v]];
        }
        s->nlev = l + 1;
        if (last) break;
        /* next level graph: groups adjacent if a fine edge joins them */
        int m = ng;
        int* pr = (int*)malloc(sizeof(int) * 2 * (ptr[n] + 1));
        int np = 0;
        for (int u = 0; u < n; ++u)
            for (int k = ptr[u]; k < ptr[u + 1]; ++k) {
                int a = s->group_of[l][u], b = s->group_of[l][nb[k]];
                if (a != b) {
                    pr[2 * np] = a;
                    pr[2 * np + 1] = b;
                    ++np;
                }
            }
        qsort(pr, np, sizeof(int) * 2, cmp_int2);
        int* ptr2 = (int*)calloc(m + 1, sizeof(int));
        int* nb2 = (int*)malloc(sizeof(int) * (np + 1));
        int na = 0;
        for (int i = 0; i < np; ++i) {
            if (i > 0 && pr[2 * i] == pr[2 * i - 2] && pr[2 * i + 1] == pr[2 * i - 1]) continue;
            nb2[na++] = pr[2 * i + 1];
            ptr2[pr[2 * i] + 1]++;
        }
        for (int i = 0; i < m; ++i) ptr2[i + 1] += ptr2[i];
        free(pr);
        free(ptr);
        free(nb);
        ptr = ptr2;
        nb = nb2;
        n = m;
    }
    free(ptr);
    free(nb);
    (void)cmp_int;
    return 0;
}

/* ---------------------------------------------------------------- scene */

OScene* o_scene_create(int nv, const double* x_rest, int nt, const int* tets,
                       const double* E, const double* nu, const double* rho,
                       const double* gravity, const double* ground,
                       const OParams* prm) {
    if (nv <= 0 || nt <= 0) {
        o_set_error("empty mesh");
        return NULL;
    }
    OScene* s = (OScene*)calloc(1, sizeof(OScene));
    s->nv = nv;
    s->nt = nt;
    s->prm = *prm;
    if (s->prm.subdomain <= 0) s->prm.subdomain = 32;
    s->x_rest = (double*)malloc(sizeof(double) * 3 * (size_t)nv);
    memcpy(s->x_rest, x_rest, sizeof(double) * 3 * (size_t)nv);
    s->tets = (int*)malloc(sizeof(int) * 4 * (size_t)nt);
    memcpy(s->tets, tets, sizeof(int) * 4 * (size_t)nt);
    for (int i = 0; i < 4 * nt; ++i)
        if (tets[i] < 0 || tets[i] >= nv) {
            o_set_error("tet index out of range");
            o_scene_destroy(s);
            return NULL;
        }
    if (o_build_mesh(s) != 0) {
        o_scene_destroy(s);
        return NULL;
    }
    for (int t = 0; t < nt; ++t) {
        s->mu[t] = E[t] / (2.0 * (1.0 + nu[t]));
        s->lam[t] = E[t] * nu[t] / ((1.0 + nu[t]) * (1.0 - 2.0 * nu[t]));
        for (int j = 0; j < 4; ++j) s->mass[tets[4 * t + j]] += 0.25 * rho[t] * s->vol[t];
    }
    for (int i = 0; i < 3; ++i) s->gravity[i] = gravity[i];
    s->has_ground = ground && !isnan(ground[3]);
    if (s->has_ground) {
        double l = sqrt(ground[0] * ground[0] + ground[1] * ground[1] + ground[2] * ground[2]);
        for (int i = 0; i < 3; ++i) s->gn[i] = ground[i] / l;
        s->goff = ground[3];
    }
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int v = 0; v < nv; ++v)
        for (int i = 0; i < 3; ++i) {
            double c = x_rest[3 * v + i];
            if (c < lo[i]) lo[i] = c;
            if (c > hi[i]) hi[i] = c;
        }
    s->bbox = sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                   (hi[2] - lo[2]) * (hi[2] - lo[2]));
    build_surface(s);
    build_adjacency(s);
    build_bodies(s);
    o_build_hierarchy(s);
    return s;
}

void o_scene_destroy(OScene* s) {
    if (!s) return;
    free(s->x_rest);
    free(s->tets);
    free(s->mu);
    free(s->lam);
    free(s->vol);
    free(s->Dm_inv);
    free(s->mass);
    free(s->sv);
    free(s->sf);
    free(s->se);
    free(s->on_surface);
    free(s->adj_ptr);
    free(s->adj);
    free(s->body);
    for (int l = 0; l < s->nlev; ++l) {
        free(s->group_of[l]);
        free(s->slot_of[l]);
        free(s->gsize[l]);
        free(s->members[l]);
        free(s->node_of_vert[l]);
        if (s->fac[l]) {
            for (int g = 0; g < s->ngroups[l]; ++g) free(s->fac[l][g]);
            free(s->fac[l]);
        }
    }
    if (s->blk0) {
        for (int g = 0; g < s->ngroups[0]; ++g) free(s->blk0[g]);
        free(s->blk0);
    }
    if (s->topk) {
        for (int g = 0; g < s->ngroups[0]; ++g) free(s->topk[g]);
        free(s->topk);
    }
    free(s->ntopk);
    free(s->upd);
    o_bsr_free(&s->Hb);
    o_clist_free(&s->cbase);
    free(s->trace);
    free(s);
}

void o_surface_counts(const OScene* s, int counts[3]) {
    counts[0] = s->nsv;
    counts[1] = s->nsf;
    counts[2] = s->nse;
}

void o_surface_get(const OScene* s, int* verts, int* tris, int* edges) {
    if (verts) memcpy(verts, s->sv, sizeof(int) * s->nsv);
    if (tris) memcpy(tris, s->sf, sizeof(int) * 3 * s->nsf);
    if (edges) memcpy(edges, s->se, sizeof(int) * 2 * s->nse);
}

void o_mass_get(const OScene* s, double* mass) { memcpy(mass, s->mass, sizeof(double) * s->nv); }

double o_bbox_diag(const OScene* s) { return s->bbox; }

int o_bodies(const OScene* s, int* body_of_vertex) {
    if (body_of_vertex) memcpy(body_of_vertex, s->body, sizeof(int) * s->nv);
    return s->nbody;
}

int o_levels(const OScene* s) { return s->nlev; }

void o_level_info(const OScene* s, int level, int* n_nodes, int* n_groups) {
    *n_nodes = s->nnodes[level];
    *n_groups = s->ngroups[level];
}

void o_level_map(const OScene* s, int level, int* group_of_node, int* slot_of_node) {
    memcpy(group_of_node, s->group_of[level], sizeof(int) * s->nnodes[level]);
    memcpy(slot_of_node, s->slot_of[level], sizeof(int) * s->nnodes[level]);
}
