/* Private declarations of the FP64 oracle (test infrastructure only). */
#ifndef IPC_ORACLE_INTERNAL_H
#define IPC_ORACLE_INTERNAL_H

#include "oracle.h"
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define O_MAX_LEVELS 8

/* One active contact (Eq. 1 barrier term, Eq. 5 rank-1 Hessian). */
typedef struct OContact {
    int type;            /* 0 PT, 1 EE, 2 PG */
    int v[4];            /* vertex ids, -1 unused */
    int ida, idb;        /* key: PT (vertex, surface tri), EE (edge i<j), PG (vertex, 0) */
    double d;            /* distance */
    double k;            /* kappa * b''(d) */
    double bp;           /* kappa * b'(d) */
    double n[12];        /* nabla d over v[0..3] */
} OContact;

typedef struct OContactList {
    OContact* c;
    int n, cap;
} OContactList;

/* Block-sparse symmetric matrix, 3x3 blocks, CSR by block row. */
typedef struct OBsr {
    int nb;              /* block rows */
    int* rp;             /* nb+1 */
    int* ci;             /* nnzb */
    double* val;         /* 9*nnzb, row-major blocks */
    int nnzb;
} OBsr;

/* One rank-1 update vector u = sqrt(dS) n_curr over at most 4 vertices. */
typedef struct OUpdate {
    int v[4];
    double u[12];
    double dS;
    int type, ida, idb;
} OUpdate;

struct OScene {
    int nv, nt;
    double* x_rest;
    int* tets;
    double *mu, *lam, *vol, *Dm_inv, *mass;
    double gravity[3];
    int has_ground;
    double gn[3], goff;
    OParams prm;
    double bbox;

    /* surface (canonical order) */
    int nsv, nsf, nse;
    int *sv, *sf, *se;
    int* on_surface;
    double cell;            /* mean rest length of surface edges (pair-search cell) */

    /* vertex adjacency from tet edges */
    int *adj_ptr, *adj;
    /* connected components of the tet mesh, numbered by lowest vertex id */
    int nbody;
    int* body;

    /* MAS hierarchy: level l nodes, grouped into subdomains of <= subdomain
     * nodes.  node_of_vert[l][v] is the level-l node containing vertex v
     * (level 0: v itself). */
    int nlev;
    int nnodes[O_MAX_LEVELS], ngroups[O_MAX_LEVELS];
    int* group_of[O_MAX_LEVELS];
    int* slot_of[O_MAX_LEVELS];
    int* gsize[O_MAX_LEVELS];
    int* members[O_MAX_LEVELS];   /* BFS order: group g = members[g*S .. g*S+gsize) */
    int* node_of_vert[O_MAX_LEVELS];

    /* restart state */
    OBsr Hb;
    OContactList cbase;
    double** blk0;          /* level-0 base blocks S_d H_base S_d^T, dense */
    double** fac[O_MAX_LEVELS];   /* coarse Cholesky factors (levels >= 1) */
    OUpdate* upd;           /* classified updates (dS > 0) */
    int nupd, capupd;
    int** topk;             /* per level-0 group: indices into upd, K each */
    int* ntopk;

    /* trace of the last step */
    OIterRecord* trace;
    int ntrace, captrace;
};

/* error */
void o_set_error(const char* fmt, ...);

/* small dense linear algebra */
int o_chol(int n, double* A);
void o_chol_solve(int n, const double* L, double* b);
void o_jacobi_eig(int n, double* A, double* evals, double* Q);

/* mesh */
int o_build_mesh(OScene* s);
int o_build_hierarchy(OScene* s);

/* contacts */
void o_clist_free(OContactList* l);
void o_find_contacts(OScene* s, const double* x, OContactList* out);
int o_contact_cmp(const void* a, const void* b);

/* pair search: overlapping boxes (6 doubles lo, hi each), sorted unique */
int o_box_pairs(int na, const double* boxA, int nb, const double* boxB, int same_set, double cs, int** out);

/* elastic */
void o_tet_gather(const OScene* s, int t, const double* x, double* x12);

/* MAS */
void o_restart(OScene* s, const double* x, const OContactList* C);
void o_classify(OScene* s, const OContactList* C);
void o_apply_P(OScene* s, const double* g, double* z);
void o_forms(OScene* s, const double* z, const double* p, double out[3]);
void o_bsr_free(OBsr* m);
void o_bsr_mul(const OBsr* m, const double* in, double* out);

#endif
