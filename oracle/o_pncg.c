/* Oracle: the incremental potential (Eq. 1), its gradient, the 2D subspace
 * solve (Eq. 10; supplement Eq. 19-22) and Algorithm 1 for one timestep.
 * Test infrastructure only.
 *
 * Readings (the paper is silent or ambiguous):
 *  - Convergence (Algorithm 1, break test): max over vertices of |z_v|_2 <=
 *    tol * h * bbox_diag, declared only on restart iterations, after the
 *    step.  When a non-restart iteration already meets it, the next
 *    iteration is forced to restart so the test is repeated with a freshly
 *    built P (otherwise a near-quadratic step keeps r_k ~ 0 and never
 *    restarts).
 *  - Restart iterations use mu = g^T z / z^T H~ z, nu = 0 (Algorithm 1); a
 *    non-positive denominator falls back to mu = 1.
 *  - 2x2 singular test |Delta| < eps_sing * max(A11 A22, eps_abs) falls back
 *    to (mu, nu) = (1, 0) (supplement Eq. 21).
 *  - r_k = |g_{k+1}^T z_k| / (g_{k+1}^T z_{k+1}) with z_0 = 0; a non-positive
 *    denominator forces a restart.
 *  - Energy check ("Line Search" stage of Table 2): the first trial is the
 *    per-subdomain step x + sum_d alpha_d S_d p; it is accepted if
 *    E(x_{k+1}) <= E(x_k) + tau, where tau bounds the rounding of the two
 *    computed energies: tau = 64 u (|E(x_k)| + 4 h^2 sum_t V_t mu_t), u =
 *    2^-52.  The second term is the size of the elastic terms before they
 *    cancel (mu/2 (|F|^2 - 3) - mu (J - 1) is a difference of O(mu) values
 *    near the rest state); inertia and barrier terms are non-negative and
 *    are covered by |E|.  Without tau, a step whose decrease is below the
 *    resolution of E is accepted or rejected by rounding alone.
 *    Per-subdomain scaling of p is not in general a descent direction (it
 *    can stretch a body whose lower subdomains are clamped), so a rejected
 *    first trial falls back to per-body steps (each
 *    connected body moves uniformly by its own verified alpha_b) scaled by
 *    1, 1/2, 1/4, 1/8 -- skipped when no body exceeds the uniform step --
 *    then to the uniform step beta = min_d alpha_d (safe by construction)
 *    halved until one is accepted, ls_max + 1 trials in all. When the
 *    per-subdomain verification of straddling pairs fell back to the
 *    uniform step and the per-body verification did not, the per-subdomain
 *    trial would be that uniform step: the per-body step (verified, and no
 *    smaller anywhere) is tried first instead, and the per-body tier goes on
 *    at 1/2, 1/4, 1/8.
 *    If none is accepted, x does not move and the next iteration restarts.
 *  - Algorithm 1 tests convergence (restart and |z| <= eps) after the update
 *    whatever the update was, so a restart iteration with |z| <= eps ends the
 *    step converged even when no trial was accepted (the remaining step is
 *    below the tolerance); a rejection on a restart iteration with |z| > eps
 *    ends the step unconverged.
 *  - Velocity update v = (x^{t+1} - x^t) / h; x~ = x + h v + h^2 gravity.
 */
#include "o_internal.h"

static double elastic_energy(OScene* s, const double* x) {
    double E = 0.0;
    for (int t = 0; t < s->nt; ++t) {
        double x12[12], e;
        o_tet_gather(s, t, x, x12);
        o_snh_tet(s->Dm_inv + 9 * t, s->vol[t], s->mu[t], s->lam[t], x12, &e, NULL, NULL, 0);
        E += e;
    }
    return E;
}

static double energy_with(OScene* s, const double* x, const double* xt, const OContactList* C) {
    double Ein = 0.0;
    for (int v = 0; v < s->nv; ++v) {
        double d2 = 0.0;
        for (int r = 0; r < 3; ++r) {
            double d = x[3 * v + r] - xt[3 * v + r];
            d2 += d * d;
        }
        Ein += 0.5 * s->mass[v] * d2;
    }
    double Eel = s->prm.h * s->prm.h * elastic_energy(s, x);
    double Eb = 0.0;
    for (int i = 0; i < C->n; ++i) {
        double b[3];
        o_barrier(C->c[i].d, s->prm.dhat, b);
        Eb += s->prm.kappa * b[0];
    }
    return Ein + Eel + Eb;
}

double o_energy_tolerance(OScene* s, double E) {
    double el = 0.0;
    for (int t = 0; t < s->nt; ++t) el += s->vol[t] * s->mu[t];
    return 64.0 * ldexp(1.0, -52) * (fabs(E) + 4.0 * s->prm.h * s->prm.h * el);
}

double o_energy(OScene* s, const double* x, const double* xtilde) {
    OContactList C = {0};
    o_find_contacts(s, x, &C);
    double E = energy_with(s, x, xtilde, &C);
    o_clist_free(&C);
    return E;
}

static void gradient_with(OScene* s, const double* x, const double* xt, const OContactList* C, double* g) {
    double h2 = s->prm.h * s->prm.h;
    for (int v = 0; v < s->nv; ++v)
        for (int r = 0; r < 3; ++r) g[3 * v + r] = s->mass[v] * (x[3 * v + r] - xt[3 * v + r]);
    for (int t = 0; t < s->nt; ++t) {
        double x12[12], g12[12];
        o_tet_gather(s, t, x, x12);
        o_snh_tet(s->Dm_inv + 9 * t, s->vol[t], s->mu[t], s->lam[t], x12, NULL, g12, NULL, 0);
        for (int j = 0; j < 4; ++j)
            for (int r = 0; r < 3; ++r) g[3 * s->tets[4 * t + j] + r] += h2 * g12[3 * j + r];
    }
    for (int i = 0; i < C->n; ++i) {
        const OContact* c = C->c + i;
        int nvv = c->type == 2 ? 1 : 4;
        for (int j = 0; j < nvv; ++j)
            for (int r = 0; r < 3; ++r) g[3 * c->v[j] + r] += c->bp * c->n[3 * j + r];
    }
}

void o_gradient(OScene* s, const double* x, const double* xtilde, double* g) {
    OContactList C = {0};
    o_find_contacts(s, x, &C);
    gradient_with(s, x, xtilde, &C, g);
    o_clist_free(&C);
}

void o_solve2x2(double A11, double A12, double A22, double b1, double b2, double eps_sing, double eps_abs,
                double* mu, double* nu) {
    double det = A11 * A22 - A12 * A12;
    double ref = A11 * A22 > eps_abs ? A11 * A22 : eps_abs;
    if (!(fabs(det) >= eps_sing * ref)) {
        *mu = 1.0;
        *nu = 0.0;
        return;
    }
    /* [A11 -A12; -A12 A22] [mu; nu] = [b1; b2] */
    *mu = (A22 * b1 + A12 * b2) / det;
    *nu = (A12 * b1 + A11 * b2) / det;
}

static double dotn(const double* a, const double* b, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void push_trace(OScene* s, const OIterRecord* r) {
    if (s->ntrace == s->captrace) {
        s->captrace = s->captrace ? 2 * s->captrace : 64;
        s->trace = (OIterRecord*)realloc(s->trace, sizeof(OIterRecord) * s->captrace);
    }
    s->trace[s->ntrace++] = *r;
}

int o_trace(const OScene* s, OIterRecord* rec, int cap) {
    int n = s->ntrace < cap ? s->ntrace : cap;
    if (rec) memcpy(rec, s->trace, sizeof(OIterRecord) * n);
    return s->ntrace;
}

int o_step(OScene* s, double* x, double* v, OStepStats* st) {
    int nv = s->nv, n3 = 3 * nv;
    double h = s->prm.h;
    double eps = s->prm.tol * h * s->bbox;
    double* xt = (double*)malloc(sizeof(double) * n3);
    double* xk = (double*)malloc(sizeof(double) * n3);
    double* xstart = (double*)malloc(sizeof(double) * n3);
    double* g = (double*)malloc(sizeof(double) * n3);
    double* z = (double*)malloc(sizeof(double) * n3);
    double* zprev = (double*)calloc(n3, sizeof(double));
    double* p = (double*)calloc(n3, sizeof(double));
    double* q = (double*)malloc(sizeof(double) * n3);
    double* xtry = (double*)malloc(sizeof(double) * n3);
    double* alpha = (double*)malloc(sizeof(double) * s->ngroups[0]);
    double* alpha_b = (double*)malloc(sizeof(double) * s->nbody);
    memcpy(xstart, x, sizeof(double) * n3);
    memcpy(xk, x, sizeof(double) * n3);
    for (int i = 0; i < nv; ++i)
        for (int r = 0; r < 3; ++r) xt[3 * i + r] = x[3 * i + r] + h * v[3 * i + r] + h * h * s->gravity[r];

    OStepStats S;
    memset(&S, 0, sizeof S);
    s->ntrace = 0;
    OContactList C = {0}, Ctry = {0};
    o_find_contacts(s, xk, &C);
    double Ek = energy_with(s, xk, xt, &C);
    int restart = 1, k;
    for (k = 0; k < s->prm.iter_max; ++k) {
        OIterRecord rec;
        memset(&rec, 0, sizeof rec);
        rec.restart = restart;
        rec.n_contacts = C.n;
        if (restart) {
            o_restart(s, xk, &C);
            S.restarts++;
        } else {
            o_classify(s, &C);
        }
        rec.n_update = s->nupd;
        gradient_with(s, xk, xt, &C, g);
        o_apply_P(s, g, z);
        double gz = dotn(g, z, n3);
        double forms[3];
        double mu, nu;
        if (restart) {
            o_forms(s, z, z, forms);
            mu = forms[0] > 0.0 ? gz / forms[0] : 1.0;
            nu = 0.0;
        } else {
            o_forms(s, z, p, forms);
            o_solve2x2(forms[0], forms[1], forms[2], gz, -dotn(g, p, n3), s->prm.eps_sing, s->prm.eps_abs, &mu,
                       &nu);
        }
        for (int i = 0; i < n3; ++i) p[i] = -mu * z[i] + nu * p[i];
        rec.mu = mu;
        rec.nu = nu;
        rec.gz = gz;
        double zn = 0.0;
        for (int i = 0; i < nv; ++i) {
            double a = sqrt(z[3 * i] * z[3 * i] + z[3 * i + 1] * z[3 * i + 1] + z[3 * i + 2] * z[3 * i + 2]);
            if (a > zn) zn = a;
        }
        rec.znorm = zn;
        S.znorm = zn;
        /* step sizes per level-0 subdomain and per body */
        int passes_b = 0;
        const int passes = o_ccd(s, xk, p, alpha, alpha_b, &passes_b);
        rec.ccd_passes = passes;
        rec.ccd_passes_body = passes_b;
        rec.alpha_min = 1.0;
        rec.alpha_max = 0.0;
        for (int gi = 0; gi < s->ngroups[0]; ++gi) {
            if (alpha[gi] < rec.alpha_min) rec.alpha_min = alpha[gi];
            if (alpha[gi] > rec.alpha_max) rec.alpha_max = alpha[gi];
        }
        double bmax = 0.0;
        for (int b = 0; b < s->nbody; ++b)
            if (alpha_b[b] > bmax) bmax = alpha_b[b];
        /* energy check over the trial list: per-subdomain step; per-body
         * steps scaled by 1, 1/2, 1/4, 1/8; uniform steps alpha_min / 2^j.
         * When the per-subdomain verification fell back to the uniform step
         * and the per-body one did not, the first trial is the per-body step
         * (also verified, and at least the uniform step everywhere), and the
         * per-body tier continues at 1/2. */
        rec.energy_before = Ek;
        int accepted = 0, halv = 0;
        int body_tier = bmax > rec.alpha_min;
        int body_first = body_tier && passes < 0 && passes_b >= 0;
        int nbody_trials = body_tier ? (body_first ? 3 : 4) : 0;
        int j0 = (rec.alpha_max > rec.alpha_min || body_tier) ? 0 : 1;
        for (int ls = 0; ls <= s->prm.ls_max; ++ls) {
            if (ls == 0 && !body_first) {
                for (int i = 0; i < nv; ++i)
                    for (int r = 0; r < 3; ++r)
                        xtry[3 * i + r] = xk[3 * i + r] + alpha[s->group_of[0][i]] * p[3 * i + r];
            } else if (ls == 0 || ls <= nbody_trials) {
                double c = ldexp(1.0, -(ls + (body_first ? 0 : -1)));
                for (int i = 0; i < nv; ++i)
                    for (int r = 0; r < 3; ++r)
                        xtry[3 * i + r] = xk[3 * i + r] + c * alpha_b[s->body[i]] * p[3 * i + r];
            } else {
                int j = j0 + (ls - 1 - nbody_trials);
                double beta = ldexp(rec.alpha_min, -j);
                for (int i = 0; i < n3; ++i) xtry[i] = xk[i] + beta * p[i];
            }
            o_find_contacts(s, xtry, &Ctry);
            double Et = energy_with(s, xtry, xt, &Ctry);
            if (Et <= Ek + o_energy_tolerance(s, Ek)) {
                accepted = 1;
                memcpy(xk, xtry, sizeof(double) * n3);
                OContactList tmp = C;
                C = Ctry;
                Ctry = tmp;
                Ek = Et;
                break;
            }
            ++halv;
        }
        rec.ls_halvings = halv;
        rec.energy_after = Ek;
        S.ls_halvings += halv;
        int forced = 0;
        if (!accepted) {
            S.ls_failures++;
            forced = 1;
        }
        if (restart && zn <= eps) {
            S.converged = 1;
            push_trace(s, &rec);
            ++k;
            break;
        }
        if (forced && restart) {
            push_trace(s, &rec);
            ++k;
            break;
        }
        double den = gz;
        double r = den > 0.0 ? fabs(dotn(g, zprev, n3)) / den : INFINITY;
        rec.r = r;
        restart = forced || !(r <= s->prm.delta) || zn <= eps;
        memcpy(zprev, z, sizeof(double) * n3);
        push_trace(s, &rec);
    }
    S.iters = k;
    S.energy = Ek;
    S.n_contacts = C.n;
    S.min_dist = INFINITY;
    for (int i = 0; i < C.n; ++i)
        if (C.c[i].d < S.min_dist) S.min_dist = C.c[i].d;
    for (int i = 0; i < n3; ++i) {
        v[i] = (xk[i] - xstart[i]) / h;
        x[i] = xk[i];
    }
    if (st) *st = S;
    o_clist_free(&C);
    o_clist_free(&Ctry);
    free(xt);
    free(xk);
    free(xstart);
    free(g);
    free(z);
    free(zprev);
    free(p);
    free(q);
    free(xtry);
    free(alpha);
    free(alpha_b);
    return S.converged ? 0 : 1;
}
