/* Oracle: H_base, the MAS preconditioner and the Sparse-Input update.
 * Test infrastructure only.
 *
 *  - H_base at a restart point x_b (Eq. 6): lumped mass + h^2 * projected
 *    SNH Hessian + sum over C_base of k n n^T (Eq. 5), assembled as a
 *    block-sparse matrix.
 *  - MAS (supplement Eq. 1-4): level-0 blocks S_d H_base S_d^T; coarse
 *    matrices A_l = C_l H_base C_l^T restricted to each level-l subdomain,
 *    where C_l sums the xyz components of the fine vertices of a cluster.
 *    Coarse inverses are factorised at the restart and frozen (Eq. 8).
 *  - Classification (Sec. 4.1.1): a current contact absent from C_base is
 *    new (u = sqrt(k) n, dS = k); a contact whose normal turned by more than
 *    eps_rot is treated as new; a stiffer one adds u = sqrt(k - k_b) n with
 *    dS = k - k_b; a softer one is ignored.  Reading: the rotation test
 *    compares the cosine of the angle between the 12-vectors n_curr, n_base
 *    with cos(eps_rot).
 *  - Localised top-K: per level-0 subdomain, the K classified vectors with
 *    the largest dS (ties by ascending contact key) whose support touches the
 *    subdomain; u_d = S_d u.
 *  - Level-0 inverse rebuilt from scratch each iteration as
 *    (S_d H_base S_d^T + U_d U_d^T)^-1 by Cholesky: the matrix the Woodbury
 *    formula of Eq. 7 inverts.
 *  - Reading: H~ = H_base + U U^T in the 2x2 forms uses every classified
 *    vector (dS > 0), not only the top-K ones.
 */
#include "o_internal.h"

/* ---------------------------------------------------------------- BSR */

typedef struct Trip {
    int r, c;
    double v[9];
} Trip;

static int trip_cmp(const void* a, const void* b) {
    const Trip* x = (const Trip*)a;
    const Trip* y = (const Trip*)b;
    if (x->r != y->r) return x->r < y->r ? -1 : 1;
    if (x->c != y->c) return x->c < y->c ? -1 : 1;
    return 0;
}

void o_bsr_free(OBsr* m) {
    free(m->rp);
    free(m->ci);
    free(m->val);
    memset(m, 0, sizeof *m);
}

void o_bsr_mul(const OBsr* m, const double* in, double* out) {
    for (int i = 0; i < m->nb; ++i) {
        double acc[3] = {0, 0, 0};
        for (int k = m->rp[i]; k < m->rp[i + 1]; ++k) {
            const double* B = m->val + 9 * (size_t)k;
            const double* y = in + 3 * m->ci[k];
            for (int r = 0; r < 3; ++r) acc[r] += B[3 * r] * y[0] + B[3 * r + 1] * y[1] + B[3 * r + 2] * y[2];
        }
        for (int r = 0; r < 3; ++r) out[3 * i + r] = acc[r];
    }
}

static void add_elem(Trip** T, int* n, int* cap, const int* v, int nvv, const double* H, int ld) {
    for (int a = 0; a < nvv; ++a)
        for (int b = 0; b < nvv; ++b) {
            if (*n == *cap) {
                *cap = *cap ? 2 * *cap : 1024;
                *T = (Trip*)realloc(*T, sizeof(Trip) * (*cap));
            }
            Trip* t = *T + (*n)++;
            t->r = v[a];
            t->c = v[b];
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) t->v[3 * r + c] = H[(3 * a + r) * ld + 3 * b + c];
        }
}

static void build_Hbase(OScene* s, const double* x, const OContactList* C, OBsr* out) {
    Trip* T = NULL;
    int n = 0, cap = 0;
    double h2 = s->prm.h * s->prm.h;
    for (int v = 0; v < s->nv; ++v) {
        double M[9] = {s->mass[v], 0, 0, 0, s->mass[v], 0, 0, 0, s->mass[v]};
        add_elem(&T, &n, &cap, &v, 1, M, 3);
    }
    /* per-tet projected Hessians (independent: computed in parallel when
     * OpenMP is on, appended in tet order either way, so the assembled
     * matrix does not depend on the thread count) */
    double* Ht = (double*)malloc(sizeof(double) * 144 * (size_t)(s->nt > 0 ? s->nt : 1));
#pragma omp parallel for schedule(static)
    for (int t = 0; t < s->nt; ++t) {
        double x12[12];
        double* Hq = Ht + 144 * (size_t)t;
        o_tet_gather(s, t, x, x12);
        o_snh_tet(s->Dm_inv + 9 * t, s->vol[t], s->mu[t], s->lam[t], x12, NULL, NULL, Hq, 1);
        for (int i = 0; i < 144; ++i) Hq[i] *= h2;
    }
    for (int t = 0; t < s->nt; ++t) add_elem(&T, &n, &cap, s->tets + 4 * t, 4, Ht + 144 * (size_t)t, 12);
    free(Ht);
    double* H = (double*)malloc(sizeof(double) * 144);
    for (int i = 0; i < C->n; ++i) {
        const OContact* c = C->c + i;
        int nvv = c->type == 2 ? 1 : 4;
        int d = 3 * nvv;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) H[a * d + b] = c->k * c->n[a] * c->n[b];
        add_elem(&T, &n, &cap, c->v, nvv, H, d);
    }
    free(H);
    qsort(T, n, sizeof(Trip), trip_cmp);
    o_bsr_free(out);
    out->nb = s->nv;
    out->rp = (int*)calloc(s->nv + 1, sizeof(int));
    out->ci = (int*)malloc(sizeof(int) * (n + 1));
    out->val = (double*)malloc(sizeof(double) * 9 * (size_t)(n + 1));
    int m = 0;
    for (int i = 0; i < n; ++i) {
        if (m > 0 && out->ci[m - 1] == T[i].c && i > 0 && T[i - 1].r == T[i].r) {
            for (int k = 0; k < 9; ++k) out->val[9 * (size_t)(m - 1) + k] += T[i].v[k];
            continue;
        }
        out->ci[m] = T[i].c;
        memcpy(out->val + 9 * (size_t)m, T[i].v, sizeof(double) * 9);
        out->rp[T[i].r + 1]++;
        ++m;
    }
    for (int v = 0; v < s->nv; ++v) out->rp[v + 1] += out->rp[v];
    out->nnzb = m;
    free(T);
}

/* dense block of level l, group g: sum over fine blocks (v,w) whose level-l
 * nodes lie in group g, placed at the nodes' slots. */
static double** level_blocks(OScene* s, int l) {
    int ng = s->ngroups[l];
    double** blk = (double**)calloc(ng, sizeof(double*));
    for (int g = 0; g < ng; ++g) {
        int m = 3 * s->gsize[l][g];
        blk[g] = (double*)calloc((size_t)m * m, sizeof(double));
    }
    const int* node = s->node_of_vert[l];
    for (int v = 0; v < s->nv; ++v) {
        int I = node[v];
        int gI = s->group_of[l][I];
        for (int k = s->Hb.rp[v]; k < s->Hb.rp[v + 1]; ++k) {
            int J = node[s->Hb.ci[k]];
            if (s->group_of[l][J] != gI) continue;
            int m = 3 * s->gsize[l][gI];
            int a = s->slot_of[l][I], b = s->slot_of[l][J];
            const double* B = s->Hb.val + 9 * (size_t)k;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) blk[gI][(3 * a + r) * m + 3 * b + c] += B[3 * r + c];
        }
    }
    return blk;
}

static void free_blocks(double** b, int n) {
    if (!b) return;
    for (int i = 0; i < n; ++i) free(b[i]);
    free(b);
}

void o_restart(OScene* s, const double* x, const OContactList* C) {
    build_Hbase(s, x, C, &s->Hb);
    /* C_base snapshot */
    o_clist_free(&s->cbase);
    s->cbase.n = s->cbase.cap = C->n;
    s->cbase.c = (OContact*)malloc(sizeof(OContact) * (C->n + 1));
    memcpy(s->cbase.c, C->c, sizeof(OContact) * C->n);
    /* level 0 base blocks */
    free_blocks(s->blk0, s->ngroups[0]);
    s->blk0 = level_blocks(s, 0);
    /* coarse factors */
    for (int l = 1; l < s->nlev; ++l) {
        free_blocks(s->fac[l], s->ngroups[l]);
        s->fac[l] = level_blocks(s, l);
#pragma omp parallel for schedule(dynamic)
        for (int g = 0; g < s->ngroups[l]; ++g) {
            int m = 3 * s->gsize[l][g];
            o_chol(m, s->fac[l][g]);
        }
    }
    s->nupd = 0;
    if (!s->topk) {
        s->topk = (int**)calloc(s->ngroups[0], sizeof(int*));
        s->ntopk = (int*)calloc(s->ngroups[0], sizeof(int));
        for (int g = 0; g < s->ngroups[0]; ++g) s->topk[g] = (int*)malloc(sizeof(int) * (s->prm.K + 1));
    }
    for (int g = 0; g < s->ngroups[0]; ++g) s->ntopk[g] = 0;
}

static const OContact* find_base(const OScene* s, const OContact* c) {
    return (const OContact*)bsearch(c, s->cbase.c, s->cbase.n, sizeof(OContact), o_contact_cmp);
}

static int upd_key_less(const OUpdate* a, const OUpdate* b) {
    if (a->type != b->type) return a->type < b->type;
    if (a->ida != b->ida) return a->ida < b->ida;
    return a->idb < b->idb;
}

void o_classify(OScene* s, const OContactList* C) {
    double cos_rot = cos(s->prm.eps_rot_deg * M_PI / 180.0);
    s->nupd = 0;
    for (int i = 0; i < C->n; ++i) {
        const OContact* c = C->c + i;
        const OContact* b = find_base(s, c);
        int dim = c->type == 2 ? 3 : 12;
        double dS, scale;
        if (!b) {
            dS = c->k;
        } else {
            double nn = 0, nb = 0, bb = 0;
            for (int j = 0; j < dim; ++j) {
                nn += c->n[j] * c->n[j];
                nb += c->n[j] * b->n[j];
                bb += b->n[j] * b->n[j];
            }
            double cosang = nb / sqrt(nn * bb);
            if (cosang < cos_rot)
                dS = c->k;
            else if (c->k > b->k)
                dS = c->k - b->k;
            else
                dS = 0.0;
        }
        if (!(dS > 0.0)) continue;
        scale = sqrt(dS);
        if (s->nupd == s->capupd) {
            s->capupd = s->capupd ? 2 * s->capupd : 256;
            s->upd = (OUpdate*)realloc(s->upd, sizeof(OUpdate) * s->capupd);
        }
        OUpdate* u = s->upd + s->nupd++;
        memset(u, 0, sizeof *u);
        for (int j = 0; j < 4; ++j) u->v[j] = c->v[j];
        for (int j = 0; j < dim; ++j) u->u[j] = scale * c->n[j];
        u->dS = dS;
        u->type = c->type;
        u->ida = c->ida;
        u->idb = c->idb;
    }
    /* top-K per level-0 subdomain by insertion into a sorted list */
    int K = s->prm.K;
    for (int g = 0; g < s->ngroups[0]; ++g) s->ntopk[g] = 0;
    for (int i = 0; i < s->nupd; ++i) {
        const OUpdate* u = s->upd + i;
        int touched[4], nt = 0;
        for (int j = 0; j < 4; ++j) {
            if (u->v[j] < 0) continue;
            int g = s->group_of[0][u->v[j]];
            int dup = 0;
            for (int q = 0; q < nt; ++q) dup |= touched[q] == g;
            if (!dup) touched[nt++] = g;
        }
        for (int q = 0; q < nt; ++q) {
            int g = touched[q];
            int* L = s->topk[g];
            int n = s->ntopk[g];
            /* position: before the first entry that ranks below u */
            int pos = n;
            for (int k = 0; k < n; ++k) {
                const OUpdate* w = s->upd + L[k];
                if (u->dS > w->dS || (u->dS == w->dS && upd_key_less(u, w))) {
                    pos = k;
                    break;
                }
            }
            if (pos >= K) continue;
            int last = n < K ? n : K - 1;
            for (int k = last; k > pos; --k) L[k] = L[k - 1];
            L[pos] = i;
            if (n < K) s->ntopk[g] = n + 1;
        }
    }
}

void o_apply_P(OScene* s, const double* g, double* z) {
    int nv = s->nv;
    memset(z, 0, sizeof(double) * 3 * (size_t)nv);
    /* level 0: (A_d + U_d U_d^T)^-1 g_d, factorised from scratch */
    int ng0 = s->ngroups[0];
    int S = s->prm.subdomain;
    /* subdomains are disjoint: each writes its own entries of z */
#pragma omp parallel for schedule(dynamic)
    for (int gi = 0; gi < ng0; ++gi) {
        int cnt = s->gsize[0][gi];
        int m = 3 * cnt;
        double* A = (double*)malloc(sizeof(double) * m * m);
        memcpy(A, s->blk0[gi], sizeof(double) * m * m);
        double* ud = (double*)malloc(sizeof(double) * m);
        for (int q = 0; q < s->ntopk[gi]; ++q) {
            const OUpdate* u = s->upd + s->topk[gi][q];
            memset(ud, 0, sizeof(double) * m);
            for (int j = 0; j < 4; ++j) {
                int v = u->v[j];
                if (v < 0 || s->group_of[0][v] != gi) continue;
                int a = s->slot_of[0][v];
                for (int r = 0; r < 3; ++r) ud[3 * a + r] += u->u[3 * j + r];
            }
            for (int a = 0; a < m; ++a)
                for (int b = 0; b < m; ++b) A[a * m + b] += ud[a] * ud[b];
        }
        free(ud);
        o_chol(m, A);
        double* rhs = (double*)calloc(m, sizeof(double));
        const int* mem = s->members[0] + (size_t)gi * S;
        for (int a = 0; a < cnt; ++a)
            for (int r = 0; r < 3; ++r) rhs[3 * a + r] = g[3 * mem[a] + r];
        o_chol_solve(m, A, rhs);
        for (int a = 0; a < cnt; ++a)
            for (int r = 0; r < 3; ++r) z[3 * mem[a] + r] += rhs[3 * a + r];
        free(rhs);
        free(A);
    }
    /* coarse levels: z += C_l^T M_l^-1 C_l g */
    for (int l = 1; l < s->nlev; ++l) {
        int nn = s->nnodes[l];
        double* r = (double*)calloc(3 * (size_t)nn, sizeof(double));
        const int* node = s->node_of_vert[l];
        for (int v = 0; v < nv; ++v)
            for (int c = 0; c < 3; ++c) r[3 * node[v] + c] += g[3 * v + c];
        double* y = (double*)calloc(3 * (size_t)nn, sizeof(double));
#pragma omp parallel for schedule(dynamic)
        for (int gi = 0; gi < s->ngroups[l]; ++gi) {
            int cnt = s->gsize[l][gi], m = 3 * cnt;
            const int* mem = s->members[l] + (size_t)gi * S;
            double* rhs = (double*)calloc(m, sizeof(double));
            for (int a = 0; a < cnt; ++a)
                for (int c = 0; c < 3; ++c) rhs[3 * a + c] = r[3 * mem[a] + c];
            o_chol_solve(m, s->fac[l][gi], rhs);
            for (int a = 0; a < cnt; ++a)
                for (int c = 0; c < 3; ++c) y[3 * mem[a] + c] = rhs[3 * a + c];
            free(rhs);
        }
        for (int v = 0; v < nv; ++v)
            for (int c = 0; c < 3; ++c) z[3 * v + c] += y[3 * node[v] + c];
        free(r);
        free(y);
    }
}

/* u^T a over the support of u */
static double u_dot(const OUpdate* u, const double* a) {
    double t = 0.0;
    for (int j = 0; j < 4; ++j) {
        if (u->v[j] < 0) continue;
        for (int r = 0; r < 3; ++r) t += u->u[3 * j + r] * a[3 * u->v[j] + r];
    }
    return t;
}

/* zH~z, zH~p, pH~p with H~ = H_base + U U^T (supplement Eq. 13-18) */
void o_forms(OScene* s, const double* z, const double* p, double out[3]) {
    int n3 = 3 * s->nv;
    double* hz = (double*)malloc(sizeof(double) * n3);
    double* hp = (double*)malloc(sizeof(double) * n3);
    o_bsr_mul(&s->Hb, z, hz);
    o_bsr_mul(&s->Hb, p, hp);
    double zz = 0, zp = 0, pp = 0;
    for (int i = 0; i < n3; ++i) {
        zz += z[i] * hz[i];
        zp += z[i] * hp[i];
        pp += p[i] * hp[i];
    }
    for (int i = 0; i < s->nupd; ++i) {
        double a = u_dot(s->upd + i, z), b = u_dot(s->upd + i, p);
        zz += a * a;
        zp += a * b;
        pp += b * b;
    }
    out[0] = zz;
    out[1] = zp;
    out[2] = pp;
    free(hz);
    free(hp);
}

/* ---------------------------------------------------------------- API */

void o_hessian_apply(OScene* s, const double* x, const double* in, double* out) {
    OContactList C = {0};
    o_find_contacts(s, x, &C);
    build_Hbase(s, x, &C, &s->Hb);
    o_bsr_mul(&s->Hb, in, out);
    o_clist_free(&C);
}

void o_precond_apply(OScene* s, const double* x_base, const double* x_curr, const double* g, double* z) {
    OContactList C = {0};
    o_find_contacts(s, x_base, &C);
    o_restart(s, x_base, &C);
    if (x_curr) {
        OContactList C2 = {0};
        o_find_contacts(s, x_curr, &C2);
        o_classify(s, &C2);
        o_clist_free(&C2);
    }
    o_apply_P(s, g, z);
    o_clist_free(&C);
}

void o_hess_forms(OScene* s, const double* x_base, const double* x_curr, const double* z, const double* p,
                  double out[3]) {
    OContactList C = {0};
    o_find_contacts(s, x_base, &C);
    o_restart(s, x_base, &C);
    if (x_curr) {
        OContactList C2 = {0};
        o_find_contacts(s, x_curr, &C2);
        o_classify(s, &C2);
        o_clist_free(&C2);
    }
    o_forms(s, z, p, out);
    o_clist_free(&C);
}

/* Classified updates of the last o_classify (through o_precond_apply or
 * o_hess_forms with x_curr): their count; up to cap of them with dS, the
 * contact key (type, ida, idb) and the 12-vector u.  Test access. */
int o_updates(const OScene* s, int cap, double* dS, int* key3, double* u12) {
    int n = s->nupd < cap ? s->nupd : cap;
    for (int i = 0; i < n; ++i) {
        const OUpdate* u = s->upd + i;
        if (dS) dS[i] = u->dS;
        if (key3) {
            key3[3 * i] = u->type;
            key3[3 * i + 1] = u->ida;
            key3[3 * i + 2] = u->idb;
        }
        if (u12)
            for (int j = 0; j < 12; ++j) u12[12 * i + j] = u->u[j];
    }
    return s->nupd;
}

/* Top-K list of level-0 subdomain g after the last o_classify: its length,
 * and up to cap update indices (into o_updates' order), best first. */
int o_topk(const OScene* s, int g, int cap, int* idx) {
    if (!s->topk || g < 0 || g >= s->ngroups[0]) return 0;
    int n = s->ntopk[g] < cap ? s->ntopk[g] : cap;
    for (int i = 0; i < n; ++i) idx[i] = s->topk[g][i];
    return s->ntopk[g];
}
