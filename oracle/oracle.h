/*
 * FP64 CPU oracle of MAS-PNCG for Incremental Potential Contact.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this code; only the tests, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs do.  It shares no code with the CUDA path.
 *
 * It is a plain, slow restatement of the method:
 *   - energy of Eq. 1 (inertia + h^2 * stable neo-Hookean + kappa * log
 *     barrier; no friction), predictor x~ of Eq. 1 / Algorithm 1 input;
 *   - brute-force contact set (PT, EE, point-ground) with d < dhat;
 *   - assembled block-sparse (CSR) Hessian H_base: mass + PSD-projected
 *     elastic Hessian + rank-1 contact terms k n n^T (Eq. 5, Eq. 6);
 *   - MAS preconditioner (Sec. 3.3, supplement Eq. 1-4) whose level-0
 *     inverses are rebuilt from scratch every iteration as
 *     (S_d H_base S_d^T + U_d U_d^T)^-1 by dense Cholesky, which is what the
 *     Woodbury update of Eq. 7 computes in exact arithmetic; coarse levels are
 *     frozen between restarts (Eq. 8);
 *   - contact classification and localized top-K (Sec. 4.1.1);
 *   - 2D subspace minimisation (Eq. 9-10, supplement Eq. 10-22);
 *   - restart criterion (Eq. 11);
 *   - per-subdomain conservative CCD with the frame-invariant bound
 *     (supplement Eq. 29, 31) and the bisection-based cubic analysis
 *     (supplement Sec. 3.4, Algorithms 1-2), brute force over all pairs;
 *   - Algorithm 1 end to end, plus an energy-decrease check.
 *
 * Readings where the paper is silent are listed beside each function.
 * Parity pins live in tests/test_oracle_*.py.
 */
#ifndef IPC_ORACLE_H
#define IPC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct OParams {
    double h;            /* timestep */
    double dhat;         /* barrier activation distance */
    double kappa;        /* barrier stiffness */
    double tol;          /* convergence: max_v |z_v| <= tol * h * bbox_diag */
    double delta;        /* restart threshold on r_k (Eq. 11) */
    double eps_rot_deg;  /* normal rotation threshold (Sec. 4.1.1) */
    double ccd_shrink;   /* s in alpha_l = (1 - s) d0 / l_tight */
    double eps_sing;     /* 2x2 singular test, relative */
    double eps_abs;      /* 2x2 singular test, absolute */
    int K;               /* top-K per subdomain */
    int iter_max;        /* PNCG iteration cap */
    int levels_max;      /* MAS levels including level 0 */
    int ls_max;          /* energy-check halvings */
    int subdomain;       /* nodes per MAS subdomain (32) */
    int brute_force;     /* 1: all-pairs loops; 0: uniform-grid pair search
                            (same pairs, faster on large scenes) */
} OParams;

typedef struct OScene OScene;

typedef struct OStepStats {
    int iters;
    int restarts;
    int ls_halvings;
    int ls_failures;
    int converged;
    int n_contacts;      /* at the end of the step */
    double energy;       /* at the end of the step */
    double min_dist;     /* over active contacts at the end of the step */
    double znorm;        /* last max_v |z_v| */
} OStepStats;

/* One record per PNCG iteration of the last o_step call. */
typedef struct OIterRecord {
    int restart;
    int n_contacts;
    int n_update;        /* classified contacts with dS > 0 */
    int ls_halvings;
    double mu, nu;
    double gz, znorm;
    double energy_before, energy_after;
    double alpha_min, alpha_max;
    double r;
    int ccd_passes;      /* per-subdomain verification passes, -1 = fell back */
    int ccd_passes_body; /* per-body verification passes, -1 = fell back */
} OIterRecord;

/* ---- scene ---------------------------------------------------------- */
OScene* o_scene_create(int nv, const double* x_rest, int nt, const int* tets,
                       const double* E, const double* nu, const double* rho,
                       const double* gravity, const double* ground,
                       const OParams* prm);
void o_scene_destroy(OScene* s);
const char* o_last_error(void);

/* surface: counts[0..2] = (#surface verts, #surface tris, #surface edges) */
void o_surface_counts(const OScene* s, int counts[3]);
void o_surface_get(const OScene* s, int* verts, int* tris, int* edges);
void o_mass_get(const OScene* s, double* mass);
double o_bbox_diag(const OScene* s);

/* MAS hierarchy: number of levels, nodes and groups per level, and for a
 * level the group and local slot of every node. */
int o_levels(const OScene* s);
void o_level_info(const OScene* s, int level, int* n_nodes, int* n_groups);
void o_level_map(const OScene* s, int level, int* group_of_node, int* slot_of_node);

/* ---- per-element pieces --------------------------------------------- */
void o_barrier(double d, double dhat, double out[3]);   /* b, b', b'' */
double o_pt_distance(const double* p, const double* t0, const double* t1,
                     const double* t2, double w[3]);
double o_ee_distance(const double* a0, const double* a1, const double* b0,
                     const double* b1, double st[2]);
void o_snh_tet(const double* Dm_inv, double vol, double mu, double lam,
               const double* x12, double* e, double* g12, double* H144,
               int project);
double o_snh_psi(const double* F, double mu, double lam);
void o_snh_dPdF(const double* F, double mu, double lam, double* H81);
void o_psd_project(int n, double* A);

/* ---- global evaluations at positions x (3*nv) ----------------------- */
double o_energy(OScene* s, const double* x, const double* xtilde);
void o_gradient(OScene* s, const double* x, const double* xtilde, double* g);

/* Contact set at x.  Returns the count; fills up to cap records:
 * type (0 PT, 1 EE, 2 PG), verts[4] (-1 unused), dist, k = kappa*b''(d),
 * grad12 = nabla d over the 4 verts (3 for PG). Sorted by key. */
int o_contacts(OScene* s, const double* x, int cap, int* type, int* verts,
               int* ids, double* dist, double* kstiff, double* grad12);

/* Matrix-free check of the assembled H_base at x (restart at x, contacts
 * at x): out = H_base * in. */
void o_hessian_apply(OScene* s, const double* x, const double* in, double* out);

/* Preconditioner: restart at x_base (H_base, C_base, coarse inverses),
 * then classify the contacts at x_curr against C_base, form U_d by top-K and
 * return z = P g.  If x_curr is NULL, no update (P = P_base). */
void o_precond_apply(OScene* s, const double* x_base, const double* x_curr,
                     const double* g, double* z);

/* Quadratic forms of H~ = H_base(x_base) + U U^T (U from x_curr). */
void o_hess_forms(OScene* s, const double* x_base, const double* x_curr,
                  const double* z, const double* p, double out[3]);

/* Classification (Sec. 4.1.1) of the last o_precond_apply / o_hess_forms
 * call with x_curr: number of updates (dS > 0); up to cap of them with dS,
 * key (type, ida, idb) and u = sqrt(dS) n_curr over the contact's 4 vertices
 * (12 doubles). */
int o_updates(const OScene* s, int cap, double* dS, int* key3, double* u12);
/* Top-K list of level-0 subdomain g after that call: its length and up to
 * cap update indices, best first (dS descending, ties by key ascending). */
int o_topk(const OScene* s, int g, int cap, int* idx);

/* Dense Cholesky with the pivot floor used for every MAS block: out = A^-1
 * (n x n, row-major); returns the pivots floored.  o_chol_floors returns the
 * pivots floored by every factorisation since the last reset (reset != 0
 * clears the count). */
int o_chol_inverse(int n, const double* A, double* out);
long long o_chol_floors(int reset);

/* Host threads (OpenMP) for the loops whose iterations are independent;
 * n <= 0 only queries.  Returns the threads now used.  Results do not depend
 * on it. */
int o_set_threads(int n);

/* Rounding allowance of the energy check at energy E (see o_step). */
double o_energy_tolerance(OScene* s, double E);

/* ---- CCD -------------------------------------------------------------- */
double o_cubic_safe(const double coef[4], double alpha_l);   /* d,c,b,a */
/* safe fraction of one PT (kind 0: p, t0, t1, t2) or EE (kind 1) pair moving
 * X + t Q, 4 x 3 doubles each */
double o_pair_safe(int kind, const double* X, const double* Q, double shrink, double dhat);
double o_safe_bisect(const double coef[4], double xs, double xu, double ys, double yu);
void o_pt_cubic(const double* x4, const double* p4, double coef[4]);
void o_ee_cubic(const double* x4, const double* p4, double coef[4]);
double o_ltight_pt(const double* p4);
double o_ltight_ee(const double* p4);
double o_loriginal_pt(const double* p4);
/* per-subdomain step sizes for direction p at x; alpha has one entry per
 * level-0 subdomain; returns number of verification passes (-1 = uniform
 * fallback was taken).  If alpha_body is not NULL it receives the same for
 * the grouping by connected body (one entry per body), with its passes in
 * *passes_body. */
int o_ccd(OScene* s, const double* x, const double* p, double* alpha, double* alpha_body, int* passes_body);
int o_bodies(const OScene* s, int* body_of_vertex);

/* ---- 2x2 subspace ----------------------------------------------------- */
void o_solve2x2(double A11, double A12, double A22, double b1, double b2,
                double eps_sing, double eps_abs, double* mu, double* nu);

/* ---- Algorithm 1: one timestep, x and v updated in place ------------ */
int o_step(OScene* s, double* x, double* v, OStepStats* st);
int o_trace(const OScene* s, OIterRecord* rec, int cap);

#ifdef __cplusplus
}
#endif
#endif
