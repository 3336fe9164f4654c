/* Oracle: uniform-grid pair search for boxes (test infrastructure only).
 *
 * Returns every pair (a, b) whose closed axis-aligned boxes overlap, sorted
 * and without duplicates -- the same set a double loop over all pairs with the
 * same box test returns.  It only speeds up the oracle on large scenes; the
 * brute-force double loop stays selectable (OParams.brute_force) and a test
 * checks both give identical contact sets and step sizes.
 */
#include "o_internal.h"

typedef struct Entry {
    long long key;
    int id;
} Entry;

static int entry_cmp(const void* a, const void* b) {
    const Entry* x = (const Entry*)a;
    const Entry* y = (const Entry*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->id > y->id) - (x->id < y->id);
}

static int pair_cmp(const void* a, const void* b) {
    const int* x = (const int*)a;
    const int* y = (const int*)b;
    if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
    return (x[1] > y[1]) - (x[1] < y[1]);
}

static long long cell_key(long long i, long long j, long long k) {
    const long long off = 1LL << 20;
    return ((i + off) << 42) | ((j + off) << 21) | (k + off);
}

static int box_overlap(const double* A, const double* B) {
    for (int r = 0; r < 3; ++r)
        if (A[3 + r] < B[r] || B[3 + r] < A[r]) return 0;
    return 1;
}

int o_box_pairs(int na, const double* boxA, int nb, const double* boxB, int same_set, double cs, int** out) {
    const long long kMaxCells = 4096;
    double inv = 1.0 / cs;
    /* bin B */
    Entry* E = NULL;
    int ne = 0, ce = 0;
    int* big = (int*)malloc(sizeof(int) * (nb + 1));
    int nbig = 0;
    for (int b = 0; b < nb; ++b) {
        const double* B = boxB + 6 * (size_t)b;
        long long i0 = (long long)floor(B[0] * inv), i1 = (long long)floor(B[3] * inv);
        long long j0 = (long long)floor(B[1] * inv), j1 = (long long)floor(B[4] * inv);
        long long k0 = (long long)floor(B[2] * inv), k1 = (long long)floor(B[5] * inv);
        long long nc = (i1 - i0 + 1) * (j1 - j0 + 1) * (k1 - k0 + 1);
        if (nc > kMaxCells) {
            big[nbig++] = b;
            continue;
        }
        for (long long i = i0; i <= i1; ++i)
            for (long long j = j0; j <= j1; ++j)
                for (long long k = k0; k <= k1; ++k) {
                    if (ne == ce) {
                        ce = ce ? 2 * ce : 4096;
                        E = (Entry*)realloc(E, sizeof(Entry) * ce);
                    }
                    E[ne].key = cell_key(i, j, k);
                    E[ne].id = b;
                    ++ne;
                }
    }
    qsort(E, ne, sizeof(Entry), entry_cmp);
    int* P = NULL;
    int np = 0, cp = 0;
#define PUSH(aa, bb)                                   \
    do {                                               \
        if (np == cp) {                                \
            cp = cp ? 2 * cp : 4096;                   \
            P = (int*)realloc(P, sizeof(int) * 2 * cp); \
        }                                              \
        P[2 * np] = (aa);                              \
        P[2 * np + 1] = (bb);                          \
        ++np;                                          \
    } while (0)
    for (int a = 0; a < na; ++a) {
        const double* A = boxA + 6 * (size_t)a;
        long long i0 = (long long)floor(A[0] * inv), i1 = (long long)floor(A[3] * inv);
        long long j0 = (long long)floor(A[1] * inv), j1 = (long long)floor(A[4] * inv);
        long long k0 = (long long)floor(A[2] * inv), k1 = (long long)floor(A[5] * inv);
        long long nc = (i1 - i0 + 1) * (j1 - j0 + 1) * (k1 - k0 + 1);
        if (nc > kMaxCells) {
            for (int b = 0; b < nb; ++b)
                if ((!same_set || b > a) && box_overlap(A, boxB + 6 * (size_t)b)) PUSH(a, b);
            continue;
        }
        for (long long i = i0; i <= i1; ++i)
            for (long long j = j0; j <= j1; ++j)
                for (long long k = k0; k <= k1; ++k) {
                    long long key = cell_key(i, j, k);
                    /* first entry with this key */
                    int lo = 0, hi = ne;
                    while (lo < hi) {
                        int mid = (lo + hi) / 2;
                        if (E[mid].key < key)
                            lo = mid + 1;
                        else
                            hi = mid;
                    }
                    for (int e = lo; e < ne && E[e].key == key; ++e) {
                        int b = E[e].id;
                        if (same_set && b <= a) continue;
                        if (box_overlap(A, boxB + 6 * (size_t)b)) PUSH(a, b);
                    }
                }
        for (int q = 0; q < nbig; ++q) {
            int b = big[q];
            if ((!same_set || b > a) && box_overlap(A, boxB + 6 * (size_t)b)) PUSH(a, b);
        }
    }
#undef PUSH
    qsort(P, np, sizeof(int) * 2, pair_cmp);
    int m = 0;
    for (int i = 0; i < np; ++i) {
        if (m > 0 && P[2 * (m - 1)] == P[2 * i] && P[2 * (m - 1) + 1] == P[2 * i + 1]) continue;
        P[2 * m] = P[2 * i];
        P[2 * m + 1] = P[2 * i + 1];
        ++m;
    }
    free(E);
    free(big);
    *out = P;
    return m;
}
