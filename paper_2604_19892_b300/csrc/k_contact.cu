// Contact detection (ComputeConstraintSet of Algorithm 1) and per-subdomain
// conservative CCD (Sec. 4.4; supplement Sec. 3) with a hashed uniform grid
// broad phase.
//
// Broad phase: stored primitives (surface triangles or edges) are binned by
// the cells their boxes cover (inflated by dhat for proximity, swept over
// [x, x + p] for CCD); a primitive covering more than kMaxCells cells, or
// overflowing the entry buffer, goes to a short "large" list tested against
// every query.  A query primitive walks its own cells; a pair found in several
// cells is kept only in the cell that holds the low corner of the two boxes'
// intersection, so each pair is processed once.  The box tests are exact, so
// the candidate set equals the brute-force one.
//
// Readings: PT pairs exclude incident triangles, EE pairs exclude edges that
// share a vertex and, for the barrier, edges parallel to sin^2 < 1e-12;
// point-ground uses the plane distance.  CCD lower bound
// alpha_l = (1 - s) d0 / l_tight (supplement Eq. 29 / 31); point-ground takes
// min(1, (1 - s) d0 / (-n.p)).  alpha_d is the minimum over candidate pairs
// touching subdomain d; pairs straddling subdomains are re-checked with the
// actual motion alpha_d(v) p_v; the subdomains of a pair whose safe fraction
// rho < 1 all take the pair's smallest alpha; after at most 8 passes with a
// violation the uniform step min_d alpha_d is taken (never below it).
#include <cooperative_groups.h>

#include <mutex>

#include "geom.cuh"
#include "kernels.h"

namespace ipcb {

namespace cg = cooperative_groups;

namespace {

constexpr int kT = 128;
constexpr int kMaxCells = 64;
// Grid queries: S threads per query primitive share its bucket entries (and
// the large-box and brute-force lists) round-robin, so one crowded
// neighbourhood is not one thread's serial walk; every entry is still visited
// by exactly one of them. Swept (CCD) and candidate-list boxes cover more
// cells and entries than the proximity boxes, so they take a whole warp.
constexpr int kSplitProx = 8;
constexpr int kSplitSwept = 32;
constexpr int kCcdPasses = 8;   // verification passes before the uniform fallback
// vflags: a violation flag per grouping and pass, then the compact-list
// length of each pass
static_assert(3 * kCcdPasses <= 32, "vflags holds 32 ints");

inline int nblk(long long n, int t = kT) { return (int)((n + t - 1) / t); }

__device__ __forceinline__ int cellc(float v, float inv) { return (int)floorf(v * inv); }

__device__ __forceinline__ unsigned long long pack_cell(int i, int j, int k) {
    const int off = 1 << 20;
    return ((unsigned long long)((unsigned)(i + off) & 0x1FFFFFu) << 42) |
           ((unsigned long long)((unsigned)(j + off) & 0x1FFFFFu) << 21) | (unsigned long long)((unsigned)(k + off) & 0x1FFFFFu);
}

__device__ __forceinline__ int bucket_of(unsigned long long c, int nb) { return (int)(mix64(c) & (unsigned long long)(nb - 1)); }

// ------------------------------------------------------- FP32 broad phase
//
// Every box and grid cell is computed in FP32 from FP32 copies of the surface
// positions (x, and x + p for CCD), each copy carrying in .w a bound on its
// rounding error. Boxes are grown by that bound, so an FP32 box contains the
// exact one and FP32 boxes that miss each other prove the exact boxes miss:
// the candidate pairs are a superset of the exact-box ones, and every pair
// then takes the FP64 tests as before (same contacts, same step bounds). B300
// runs FP64 at a small fraction of its FP32 rate, and the broad phase visits
// every neighbour of every primitive.

// FP32 copies of the surface positions at x and at x + p (x again without p)
template <class R>
__global__ void k_vert_f32(Dev<R> D, const double* __restrict__ x, const R* __restrict__ p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D.nsv) return;
    const int v = D.sv[i];
    const double a0 = x[3 * v], a1 = x[3 * v + 1], a2 = x[3 * v + 2];
    float4 f = make_float4((float)a0, (float)a1, (float)a2, 0.f);
    float m = fmaxf(fabsf(f.x), fmaxf(fabsf(f.y), fabsf(f.z)));
    float4 g = f;
    if (p) {
        g = make_float4((float)(a0 + (double)p[3 * v]), (float)(a1 + (double)p[3 * v + 1]),
                        (float)(a2 + (double)p[3 * v + 2]), 0.f);
        m = fmaxf(m, fmaxf(fabsf(g.x), fmaxf(fabsf(g.y), fabsf(g.z))));
    }
    // rounding to FP32 moves a coordinate by at most 2^-24 of its size; the
    // bound covers that and the FP32 arithmetic on boxes and distances
    const float e = 4e-7f * m + 1e-30f;
    f.w = e;
    g.w = e;
    D.xf[v] = f;
    D.xpf[v] = g;
}

// FP32 box of the primitive with vertices vid[0..n) over [x, x + p], grown by
// infl (rounded up by the caller) and by the vertices' error bounds
template <class R>
__device__ __forceinline__ void prim_box(const Dev<R>& D, const int* vid, int n, float infl, float lo[3], float hi[3]) {
    float e = 0.f;
    lo[0] = lo[1] = lo[2] = 3.0e38f;
    hi[0] = hi[1] = hi[2] = -3.0e38f;
    for (int k = 0; k < n; ++k) {
        const float4 a = D.xf[vid[k]], b = D.xpf[vid[k]];
        lo[0] = fminf(lo[0], fminf(a.x, b.x));
        lo[1] = fminf(lo[1], fminf(a.y, b.y));
        lo[2] = fminf(lo[2], fminf(a.z, b.z));
        hi[0] = fmaxf(hi[0], fmaxf(a.x, b.x));
        hi[1] = fmaxf(hi[1], fmaxf(a.y, b.y));
        hi[2] = fmaxf(hi[2], fmaxf(a.z, b.z));
        e = fmaxf(e, a.w);
    }
    const float g = infl + e;
    for (int r = 0; r < 3; ++r) {
        lo[r] -= g;
        hi[r] += g;
    }
}

template <class R>
__device__ __forceinline__ void load_box(const Dev<R>& D, int j, float lo[3], float hi[3]) {
    const float4 a = D.pbox[2 * (size_t)j], b = D.pbox[2 * (size_t)j + 1];
    lo[0] = a.x;
    lo[1] = a.y;
    lo[2] = a.z;
    hi[0] = b.x;
    hi[1] = b.y;
    hi[2] = b.z;
}

__device__ __forceinline__ bool overlap(const float* lo1, const float* hi1, const float* lo2, const float* hi2) {
    return !(hi1[0] < lo2[0] || hi2[0] < lo1[0] || hi1[1] < lo2[1] || hi2[1] < lo1[1] || hi1[2] < lo2[2] ||
             hi2[2] < lo1[2]);
}

// cell indices of the box fit in int (and the box is finite)
__device__ __forceinline__ bool box_in_range(const float* lo, const float* hi, float inv) {
    bool ok = true;
    for (int r = 0; r < 3; ++r) ok &= fabsf(lo[r] * inv) < 1e9f && fabsf(hi[r] * inv) < 1e9f;
    return ok;
}

// Lower bound on the distance of pair v (PT: p, t0, t1, t2; EE: a0, a1, b0,
// b1) from the FP32 positions: FP32 distance of the differences to vertex 0,
// less a margin for the closest-point arithmetic (1e-6 of the squared local
// extent, as the FP64 test would see it) and twice the position error bound.
template <class R>
__device__ __forceinline__ float pair_dist_lb(const Dev<R>& D, int kind, const int v[4]) {
    const float4 o = D.xf[v[0]];
    f3 P[4];
    float L = 0.f, e = o.w;
    for (int j = 0; j < 4; ++j) {
        const float4 q = D.xf[v[j]];
        P[j] = {q.x - o.x, q.y - o.y, q.z - o.z};
        L = fmaxf(L, fmaxf(fabsf(P[j].x), fmaxf(fabsf(P[j].y), fabsf(P[j].z))));
        e = fmaxf(e, q.w);
    }
    const float d2 = kind == 0 ? pt_dist2_f(P[0], P[1], P[2], P[3]) : ee_dist2_f(P[0], P[1], P[2], P[3]);
    const float m = d2 - 1e-6f * L * L;
    if (!(m > 0.f)) return 0.f;
    return fmaxf(0.999f * sqrtf(m) - 2.f * e, 0.f);
}

// Visits every stored primitive j whose box overlaps the query box once:
// the query walks its own cells and keeps a pair only in the cell holding
// the low corner of the two boxes' intersection; boxes too large for the
// grid are in a short list, and a query box too large for it scans all
// nstored. Thread sub of S takes every S-th entry.
template <int S, class R, class F>
__device__ __forceinline__ void grid_query(const Dev<R>& D, const float lo[3], const float hi[3], int nstored, int sub,
                                           F&& visit) {
    const float inv = *D.cellinv;
    const int i0 = cellc(lo[0], inv), j0 = cellc(lo[1], inv), k0 = cellc(lo[2], inv);
    const int i1 = cellc(hi[0], inv), j1 = cellc(hi[1], inv), k1 = cellc(hi[2], inv);
    long long nc = ((long long)i1 - i0 + 1) * ((long long)j1 - j0 + 1) * ((long long)k1 - k0 + 1);
    if (!(nc > 0) || !box_in_range(lo, hi, inv)) nc = kMaxCells + 1;
    float blo[3], bhi[3];
    if (nc > kMaxCells) {
        for (int j = sub; j < nstored; j += S) {
            load_box(D, j, blo, bhi);
            if (overlap(lo, hi, blo, bhi)) visit(j);
        }
        return;
    }
    for (int a = i0; a <= i1; ++a)
        for (int bb = j0; bb <= j1; ++bb)
            for (int c = k0; c <= k1; ++c) {
                const unsigned long long cc = pack_cell(a, bb, c);
                const int bk = bucket_of(cc, D.nbuckets);
                for (int e = D.gstart[bk] + sub; e < D.gstart[bk + 1]; e += S) {
                    if (D.gcell[e] != cc) continue;
                    // the entry carries its box: consecutive entries are
                    // consecutive in memory, no gather through the id
                    const float4 ea = D.gbox[2 * (size_t)e], eb = D.gbox[2 * (size_t)e + 1];
                    const int j = __float_as_int(ea.w);
                    blo[0] = ea.x;
                    blo[1] = ea.y;
                    blo[2] = ea.z;
                    bhi[0] = eb.x;
                    bhi[1] = eb.y;
                    bhi[2] = eb.z;
                    if (!overlap(lo, hi, blo, bhi)) continue;
                    if (cellc(fmaxf(lo[0], blo[0]), inv) != a || cellc(fmaxf(lo[1], blo[1]), inv) != bb ||
                        cellc(fmaxf(lo[2], blo[2]), inv) != c)
                        continue;
                    visit(j);
                }
            }
    const int nl = *D.gnlarge;
    for (int k = sub; k < nl; k += S) {
        const int j = D.glarge[k];
        load_box(D, j, blo, bhi);
        if (overlap(lo, hi, blo, bhi)) visit(j);
    }
}

// infl as FP32, never below the FP64 value
__host__ inline float round_up_f(double v) {
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, 3.0e38f);
    return f;
}

// ---------------------------------------------------------------- grid build

template <class R>
__global__ void k_grid_count(Dev<R> D, const int* prims, int nper, int nprim, float infl, int* gin) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nprim) return;
    int vid[3];
    for (int k = 0; k < nper; ++k) vid[k] = prims[nper * i + k];
    float lo[3], hi[3];
    prim_box(D, vid, nper, infl, lo, hi);
    D.pbox[2 * (size_t)i] = make_float4(lo[0], lo[1], lo[2], 0.f);
    D.pbox[2 * (size_t)i + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    const float inv = *D.cellinv;
    // a box outside the cell-index range (or not finite) goes to the large list
    const bool finite = box_in_range(lo, hi, inv);
    long long n0 = finite ? (long long)cellc(hi[0], inv) - cellc(lo[0], inv) + 1 : kMaxCells + 1;
    long long n1 = finite ? (long long)cellc(hi[1], inv) - cellc(lo[1], inv) + 1 : kMaxCells + 1;
    long long n2 = finite ? (long long)cellc(hi[2], inv) - cellc(lo[2], inv) + 1 : kMaxCells + 1;
    long long nc = n0 * n1 * n2;
    bool in_grid = finite && n0 >= 1 && n1 >= 1 && n2 >= 1 && nc <= kMaxCells && n0 <= kMaxCells &&
                   n1 <= kMaxCells && n2 <= kMaxCells;
    if (in_grid) {
        int old = atomicAdd(D.gtotal, (int)nc);
        if (old + nc > D.gcap) in_grid = false;
    }
    gin[i] = in_grid ? 1 : 0;
    if (!in_grid) {
        int k = atomicAdd(D.gnlarge, 1);
        D.glarge[k] = i;
        return;
    }
    int i0 = cellc(lo[0], inv), j0 = cellc(lo[1], inv), k0 = cellc(lo[2], inv);
    for (int a = 0; a < n0; ++a)
        for (int b = 0; b < n1; ++b)
            for (int c = 0; c < n2; ++c) atomicAdd(&D.gcount[bucket_of(pack_cell(i0 + a, j0 + b, k0 + c), D.nbuckets)], 1);
}

template <class R>
__global__ void k_grid_fill(Dev<R> D, int nprim, const int* gin) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nprim || !gin[i]) return;
    float lo[3], hi[3];
    load_box(D, i, lo, hi);
    const float inv = *D.cellinv;
    int i0 = cellc(lo[0], inv), j0 = cellc(lo[1], inv), k0 = cellc(lo[2], inv);
    int i1 = cellc(hi[0], inv), j1 = cellc(hi[1], inv), k1 = cellc(hi[2], inv);
    for (int a = i0; a <= i1; ++a)
        for (int b = j0; b <= j1; ++b)
            for (int c = k0; c <= k1; ++c) {
                unsigned long long cc = pack_cell(a, b, c);
                int bk = bucket_of(cc, D.nbuckets);
                int pos = D.gstart[bk] + atomicAdd(&D.gfill[bk], 1);
                D.gbox[2 * (size_t)pos] = make_float4(lo[0], lo[1], lo[2], __int_as_float(i));
                D.gbox[2 * (size_t)pos + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
                D.gcell[pos] = cc;
            }
}

template <class R>
__global__ void k_set_cell(Dev<R> D, int ccd) {
    double cs = D.cell;
    if (ccd) cs = fmax(cs, D.S->pmax);
    else cs = fmax(cs, 2.0 * D.dhat);
    *D.cellsz = cs;
    *D.cellinv = (float)(1.0 / cs);
}

template <class R>
void build_grid(const Dev<R>& D, const int* prims, int nper, int nprim, float infl, int* gin, bool ccd, cudaStream_t st) {
    cudaMemsetAsync(D.gcount, 0, sizeof(int) * (D.nbuckets + 1), st);
    cudaMemsetAsync(D.gfill, 0, sizeof(int) * D.nbuckets, st);
    cudaMemsetAsync(D.gtotal, 0, sizeof(int), st);
    cudaMemsetAsync(D.gnlarge, 0, sizeof(int), st);
    KL(k_set_cell<R><<<1, 1, 0, st>>>(D, ccd ? 1 : 0));
    if (nprim > 0) KL(k_grid_count<R><<<nblk(nprim), kT, 0, st>>>(D, prims, nper, nprim, infl, gin));
    scan_exclusive(D.gcount, D.gstart, D.nbuckets, D.gtmp, st);
    if (nprim > 0) KL(k_grid_fill<R><<<nblk(nprim), kT, 0, st>>>(D, nprim, gin));
}

// Appends (a, b) to list (warp-aggregated); false when the list is full and
// the pair was not stored.
__device__ __forceinline__ bool append_ok(int2* list, int* count, int cap, int a, int b) {
    const unsigned m = __activemask();
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    const int rank = __popc(m & ((1u << lane) - 1u));
    int base = cap;
    if (lane == leader && *(volatile int*)count < cap) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(m, base, leader);
    const int k = base + rank;
    if (k >= cap) return false;
    list[k] = make_int2(a, b);
    return true;
}

// ------------------------------------------------------------ contact write

__device__ __forceinline__ void put_contact(const ContactBuf& C, int cap, int type, int4 v, unsigned long long key,
                                            double d, double kap, double dhat, d3 r, const double w[4], Scalars* S) {
    // counters stop growing once full (checked before the increment), so
    // they stay far below INT_MAX however many pairs qualify
    if (*(volatile int*)C.count >= cap) {
        atomicOr(&S->overflow, 1);
        return;
    }
    int i = atomicAdd(C.count, 1);
    if (i >= cap) {
        atomicOr(&S->overflow, 1);
        return;
    }
    double b, b1, b2;
    barrier3(d, dhat, b, b1, b2);
    C.type[i] = type;
    C.v[i] = v;
    C.key[i] = key;
    C.d[i] = d;
    C.k[i] = kap * b2;
    C.bp[i] = kap * b1;
    C.r[3 * i] = r.x;
    C.r[3 * i + 1] = r.y;
    C.r[3 * i + 2] = r.z;
    for (int j = 0; j < 4; ++j) C.w[4 * i + j] = w[j];
    if (d > 0.0)
        atomicMinPos(&S->min_dist, d);
    else
        S->nonpos = 1;  // touching or penetrating (bit-pattern min is only valid for d > 0)
}

// The FP32 prefilters of pt_try / ee_try: false when the pair cannot be
// within dhat (or shares a vertex), so the FP64 test is not needed.
template <class R>
__device__ __forceinline__ bool pt_needed(const Dev<R>& D, int pv, int f) {
    const int v[4] = {pv, D.sf[3 * f], D.sf[3 * f + 1], D.sf[3 * f + 2]};
    if (pv == v[1] || pv == v[2] || pv == v[3]) return false;
    return pair_dist_lb(D, 0, v) < D.dhat;
}
template <class R>
__device__ __forceinline__ bool ee_needed(const Dev<R>& D, int i, int j) {
    const int v[4] = {D.se[2 * i], D.se[2 * i + 1], D.se[2 * j], D.se[2 * j + 1]};
    if (v[0] == v[2] || v[0] == v[3] || v[1] == v[2] || v[1] == v[3]) return false;
    return pair_dist_lb(D, 1, v) < D.dhat;
}

template <class R>
__device__ void pt_try(const Dev<R>& D, const double* x, const ContactBuf& C, int pv, int f) {
    int t0 = D.sf[3 * f], t1 = D.sf[3 * f + 1], t2 = D.sf[3 * f + 2];
    if (pv == t0 || pv == t1 || pv == t2) return;
    {
        const int v[4] = {pv, t0, t1, t2};
        if (pair_dist_lb(D, 0, v) >= D.dhat) return;  // FP32 prefilter
    }
    d3 P = ld3(x + 3 * pv), A = ld3(x + 3 * t0), B = ld3(x + 3 * t1), Cc = ld3(x + 3 * t2);
    double w[3];
    double d2 = pt_closest(P, A, B, Cc, w);
    if (!(d2 < D.dhat * D.dhat)) return;
    double d = sqrt(d2);
    if (!(d < D.dhat)) return;
    d3 q = w[0] * A + w[1] * B + w[2] * Cc;
    d3 r = (1.0 / d) * (P - q);
    double ww[4] = {1.0, -w[0], -w[1], -w[2]};
    put_contact(C, D.cap, 0, make_int4(pv, t0, t1, t2), contact_key(0, pv, f), d, D.kappa, D.dhat, r, ww, D.S);
}

template <class R>
__device__ void ee_try(const Dev<R>& D, const double* x, const ContactBuf& C, int i, int j) {
    int a0 = D.se[2 * i], a1 = D.se[2 * i + 1], b0 = D.se[2 * j], b1 = D.se[2 * j + 1];
    if (a0 == b0 || a0 == b1 || a1 == b0 || a1 == b1) return;
    {
        const int v[4] = {a0, a1, b0, b1};
        if (pair_dist_lb(D, 1, v) >= D.dhat) return;  // FP32 prefilter
    }
    d3 A0 = ld3(x + 3 * a0), A1 = ld3(x + 3 * a1), B0 = ld3(x + 3 * b0), B1 = ld3(x + 3 * b1);
    d3 u = A1 - A0, v = B1 - B0;
    d3 cr = cross(u, v);
    if (dot(cr, cr) < 1e-12 * dot(u, u) * dot(v, v)) return;
    double s, t;
    double d2 = ee_closest(A0, A1, B0, B1, s, t);
    if (!(d2 < D.dhat * D.dhat)) return;
    double d = sqrt(d2);
    if (!(d < D.dhat)) return;
    d3 c1 = A0 + s * u, c2 = B0 + t * v;
    d3 r = (1.0 / d) * (c1 - c2);
    double ww[4] = {1.0 - s, s, -(1.0 - t), -t};
    put_contact(C, D.cap, 1, make_int4(a0, a1, b0, b1), contact_key(1, i, j), d, D.kappa, D.dhat, r, ww, D.S);
}

// ------------------------------------------------------------ proximity

// Grid queries. kFused = false (the default pass): a query screens every
// pair it finds in FP32 and appends the ones that need the FP64 test to the
// scratch list gpair, which the list kernels finish one thread per pair; a
// full list sets gpair_n[1]. The query kernel then holds no FP64 code, so its
// chains of dependent grid loads run at full occupancy. kFused = true: the
// query runs the FP64 test itself, grid-stride, and only when the list
// overflowed (the list kernels then skip it), so every pair is handled once.
template <class R, bool kFused>
__global__ void __launch_bounds__(kT, kFused ? 1 : 8) k_prox_pt(Dev<R> D, const double* __restrict__ x, ContactBuf C) {
    if (kFused && !D.gpair_n[1]) return;
    const long long n = (long long)D.nsv * kSplitProx;
    for (long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x; gid < n;
         gid += (long long)gridDim.x * blockDim.x) {
        const int qi = (int)(gid / kSplitProx), sub = (int)(gid % kSplitProx);
        const int pv = D.sv[qi];
        float lo[3], hi[3];
        prim_box(D, &pv, 1, 0.f, lo, hi);
        grid_query<kSplitProx>(D, lo, hi, D.nsf, sub, [&](int f) {
            if constexpr (kFused)
                pt_try(D, x, C, pv, f);
            else if (pt_needed(D, pv, f) && !append_ok(D.gpair, D.gpair_n, D.gpair_cap, pv, f))
                D.gpair_n[1] = 1;
        });
    }
}

template <class R, bool kFused>
__global__ void __launch_bounds__(kT, kFused ? 1 : 8) k_prox_ee(Dev<R> D, const double* __restrict__ x, ContactBuf C) {
    if (kFused && !D.gpair_n[1]) return;
    const long long n = (long long)D.nse * kSplitProx;
    for (long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x; gid < n;
         gid += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(gid / kSplitProx), sub = (int)(gid % kSplitProx);
        const int vid[2] = {D.se[2 * i], D.se[2 * i + 1]};
        float lo[3], hi[3];
        prim_box(D, vid, 2, 0.f, lo, hi);
        grid_query<kSplitProx>(D, lo, hi, D.nse, sub, [&](int j) {
            if (j <= i) return;
            if constexpr (kFused)
                ee_try(D, x, C, i, j);
            else if (ee_needed(D, i, j) && !append_ok(D.gpair, D.gpair_n, D.gpair_cap, i, j))
                D.gpair_n[1] = 1;
        });
    }
}

template <class R>
__global__ void k_prox_pg(Dev<R> D, const double* __restrict__ x, ContactBuf C) {
    int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= D.nsv || !D.has_ground) return;
    int pv = D.sv[qi];
    d3 n = mk(D.gn[0], D.gn[1], D.gn[2]);
    double d = dot(n, ld3(x + 3 * pv)) - D.goff;
    if (!(d < D.dhat)) return;
    double ww[4] = {1.0, 0.0, 0.0, 0.0};
    put_contact(C, D.cap, 2, make_int4(pv, -1, -1, -1), contact_key(2, pv, 0), d, D.kappa, D.dhat, n, ww, D.S);
}

template <class R>
__global__ void k_reset_detect(Dev<R> D, ContactBuf C) {
    *C.count = 0;
    D.S->min_dist = __longlong_as_double(0x7ff0000000000000ULL);
    D.S->nonpos = 0;
}

// ------------------------------------------------------------------- CCD

// distance of the pair at X + t Q (PT: p, t0, t1, t2; EE: a0, a1, b0, b1)
__device__ __forceinline__ double pair_dist_at(int kind, const d3 X[4], const d3 Q[4], double t) {
    d3 Y[4];
    for (int j = 0; j < 4; ++j) Y[j] = X[j] + t * Q[j];
    if (kind == 0) {
        double w[3];
        return sqrt(pt_closest(Y[0], Y[1], Y[2], Y[3], w));
    }
    double s, u;
    return sqrt(ee_closest(Y[0], Y[1], Y[2], Y[3], s, u));
}

template <class R>
__device__ double pair_alpha(const Dev<R>& D, int kind, const int v[4], const double* x, const R* p, const double* scale,
                             const int* grp = nullptr) {
    d3 X[4], Q[4];
    for (int j = 0; j < 4; ++j) {
        X[j] = ld3(x + 3 * v[j]);
        double s = scale ? scale[grp[v[j]]] : 1.0;
        Q[j] = mk(s * (double)p[3 * v[j]], s * (double)p[3 * v[j] + 1], s * (double)p[3 * v[j] + 2]);
    }
    // l: the largest relative displacement, one square root of the largest
    // square (the same value as the largest root: sqrt is monotone and
    // correctly rounded; FP64 square roots are costly here)
    double d0, l2 = 0.0, c[4];
    if (kind == 0) {  // (p, t0, t1, t2)
        double w[3];
        d0 = sqrt(pt_closest(X[0], X[1], X[2], X[3], w));
        for (int j = 1; j < 4; ++j) {
            d3 dd = Q[0] - Q[j];
            l2 = fmax(l2, dot(dd, dd));
        }
        cubic_of(X[2] - X[1], Q[2] - Q[1], X[3] - X[1], Q[3] - Q[1], X[0] - X[1], Q[0] - Q[1], c);
    } else {  // (a0, a1, b0, b1)
        double s, t;
        d0 = sqrt(ee_closest(X[0], X[1], X[2], X[3], s, t));
        for (int i = 0; i < 2; ++i)
            for (int j = 2; j < 4; ++j) {
                d3 dd = Q[i] - Q[j];
                l2 = fmax(l2, dot(dd, dd));
            }
        cubic_of(X[2] - X[0], Q[2] - Q[0], X[1] - X[0], Q[1] - Q[0], X[3] - X[0], Q[3] - Q[0], c);
    }
    const double l = sqrt(l2);
    double al = l > 0.0 ? (1.0 - D.ccd_shrink) * d0 / l : __longlong_as_double(0x7ff0000000000000ULL);
    double a = cubic_safe(c, al);
    // the coplanarity walk only rules out crossing; a step ending closer than
    // s min(d0, dhat) is cut back by 12 bisections between alpha_l (where
    // d >= s d0 holds) and the walk's result
    if (a > al) {
        const double thr = D.ccd_shrink * fmin(d0, D.dhat);
        if (pair_dist_at(kind, X, Q, a) < thr) {
            double lo = al > 0.0 ? al : 0.0, hi = a;
            for (int it = 0; it < 12; ++it) {
                double mid = 0.5 * (lo + hi);
                if (pair_dist_at(kind, X, Q, mid) >= thr)
                    lo = mid;
                else
                    hi = mid;
            }
            a = lo;
        }
    }
    return a;
}

// FP32 screen of a CCD pair. A pair whose distance exceeds any relative
// displacement the step can make, with every vertex scaled anywhere in
// [0, 1], keeps alpha = 1 and can never be violated by mixed per-subdomain
// steps: 0, nothing to do (FP32 lower bound on d0, sum of the two
// primitives' largest |p|).
//
// Otherwise its own step bound alpha_l = (1 - s) d0 / l uses l, the largest
// relative displacement between a vertex of one primitive and one of the
// other: where FP32 bounds already give d0 (1 - s) > l, the FP64 walk would
// return exactly 1 (CUBICSAFE starts at alpha_l >= 1), so it is not run (1).
// A pair inside one subdomain and one body moves with one common scale t in
// [0, 1] under every step the line search tries (per subdomain, per body,
// uniform), so that bound alone also keeps it safe and it needs no
// verification (0). 2: the FP64 walk is needed.
template <class R>
__device__ int ccd_screen(const Dev<R>& D, int kind, const int v[4], bool one_scale) {
    float P[4][3];
    float pa = 0.f, pb = 0.f;
    for (int j = 0; j < 4; ++j) {
        const R* q = D.p + 3 * v[j];
        P[j][0] = (float)q[0];
        P[j][1] = (float)q[1];
        P[j][2] = (float)q[2];
        float m = sqrtf(P[j][0] * P[j][0] + P[j][1] * P[j][1] + P[j][2] * P[j][2]);
        if ((kind == 0 && j == 0) || (kind == 1 && j < 2))
            pa = fmaxf(pa, m);
        else
            pb = fmaxf(pb, m);
    }
    const float lim = pair_dist_lb(D, kind, v) * (1.f - (float)D.ccd_shrink);
    if (lim > 1.001f * (pa + pb)) return 0;
    // primitive A: vertex 0 (PT) or 0, 1 (EE); B: the rest
    float lr = 0.f;
    for (int i = 0; i < (kind == 0 ? 1 : 2); ++i)
        for (int j = (kind == 0 ? 1 : 2); j < 4; ++j) {
            const float dx = P[i][0] - P[j][0], dy = P[i][1] - P[j][1], dz = P[i][2] - P[j][2];
            lr = fmaxf(lr, sqrtf(dx * dx + dy * dy + dz * dz));
        }
    // FP32 rounding of p and of the differences: a margin of 1e-3 of the
    // absolute displacements covers it many times over
    const bool whole_step = lim > 1.001f * lr + 1e-3f * (pa + pb);
    if (whole_step) return one_scale ? 0 : 1;
    return 2;
}

template <class R>
__device__ __forceinline__ bool one_scale_of(const Dev<R>& D, const int v[4]) {
    const int g0 = D.grp0[v[0]], b0 = D.body[v[0]];
    return D.grp0[v[1]] == g0 && D.grp0[v[2]] == g0 && D.grp0[v[3]] == g0 && D.body[v[1]] == b0 &&
           D.body[v[2]] == b0 && D.body[v[3]] == b0;
}

// true when ccd_pair would do more than the FP32 screen
template <class R>
__device__ __forceinline__ bool ccd_needed(const Dev<R>& D, int kind, const int v[4]) {
    return ccd_screen(D, kind, v, one_scale_of(D, v)) != 0;
}

// defer = (a, b) != nullptr: the screening pass of a cached list. A pair
// that needs the FP64 walk is appended to the scratch list gpair as (a, b)
// instead, for a second pass in which every lane of a warp runs the walk;
// when the list is full it is handled here. Every other pair is finished
// here either way.
template <class R>
__device__ void ccd_pair(const Dev<R>& D, int kind, const int v[4], const int2* defer = nullptr) {
    const int g0 = D.grp0[v[0]], g1 = D.grp0[v[1]], g2 = D.grp0[v[2]], g3 = D.grp0[v[3]];
    const int b0 = D.body[v[0]], b1 = D.body[v[1]], b2 = D.body[v[2]], b3 = D.body[v[3]];
    const bool one_scale = g1 == g0 && g2 == g0 && g3 == g0 && b1 == b0 && b2 == b0 && b3 == b0;
    const int scr = ccd_screen(D, kind, v, one_scale);
    if (scr == 0) return;
    if (scr == 2 && defer && append_ok(D.gpair, D.gpair_n, D.gpair_cap, defer->x, defer->y)) return;
    const bool whole_step = scr == 1;
    const double a = whole_step ? 1.0 : pair_alpha(D, kind, v, D.x, D.p, nullptr);
    if (a < 1.0) {
        atomicMinPos(&D.alpha[g0], a);
        if (g1 != g0) atomicMinPos(&D.alpha[g1], a);
        if (g2 != g0 && g2 != g1) atomicMinPos(&D.alpha[g2], a);
        if (g3 != g0 && g3 != g1 && g3 != g2) atomicMinPos(&D.alpha[g3], a);
        atomicMinPos(&D.alpha_b[b0], a);
        if (b1 != b0) atomicMinPos(&D.alpha_b[b1], a);
        if (b2 != b0 && b2 != b1) atomicMinPos(&D.alpha_b[b2], a);
        if (b3 != b0 && b3 != b1 && b3 != b2) atomicMinPos(&D.alpha_b[b3], a);
    }
    // keep every pair that straddles subdomains or bodies for verification
    if (!one_scale) {
        int k = *(volatile int*)&D.S->n_straddle < D.straddle_cap ? atomicAdd(&D.S->n_straddle, 1) : D.straddle_cap;
        if (k < D.straddle_cap) {
            D.str_v[k] = make_int4(v[0], v[1], v[2], v[3]);
            D.str_t[k] = kind;
        } else {
            atomicOr(&D.S->overflow, 2);
        }
    }
}

template <class R, bool kFused>
__global__ void __launch_bounds__(kT, kFused ? 1 : 7) k_ccd_pt(Dev<R> D) {
    if (kFused && !D.gpair_n[1]) return;
    const long long n = (long long)D.nsv * kSplitSwept;
    for (long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x; gid < n;
         gid += (long long)gridDim.x * blockDim.x) {
        const int qi = (int)(gid / kSplitSwept), sub = (int)(gid % kSplitSwept);
        const int pv = D.sv[qi];
        float lo[3], hi[3];
        prim_box(D, &pv, 1, 0.f, lo, hi);
        grid_query<kSplitSwept>(D, lo, hi, D.nsf, sub, [&](int f) {
            int v[4] = {pv, D.sf[3 * f], D.sf[3 * f + 1], D.sf[3 * f + 2]};
            if (pv == v[1] || pv == v[2] || pv == v[3]) return;
            if constexpr (kFused)
                ccd_pair(D, 0, v);
            else if (ccd_needed(D, 0, v) && !append_ok(D.gpair, D.gpair_n, D.gpair_cap, pv, f))
                D.gpair_n[1] = 1;
        });
    }
}

template <class R, bool kFused>
__global__ void __launch_bounds__(kT, kFused ? 1 : 7) k_ccd_ee(Dev<R> D) {
    if (kFused && !D.gpair_n[1]) return;
    const long long n = (long long)D.nse * kSplitSwept;
    for (long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x; gid < n;
         gid += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(gid / kSplitSwept), sub = (int)(gid % kSplitSwept);
        const int vid[2] = {D.se[2 * i], D.se[2 * i + 1]};
        float lo[3], hi[3];
        prim_box(D, vid, 2, 0.f, lo, hi);
        grid_query<kSplitSwept>(D, lo, hi, D.nse, sub, [&](int j) {
            if (j <= i) return;
            int v[4] = {vid[0], vid[1], D.se[2 * j], D.se[2 * j + 1]};
            if (v[0] == v[2] || v[0] == v[3] || v[1] == v[2] || v[1] == v[3]) return;
            if constexpr (kFused)
                ccd_pair(D, 1, v);
            else if (ccd_needed(D, 1, v) && !append_ok(D.gpair, D.gpair_n, D.gpair_cap, i, j))
                D.gpair_n[1] = 1;
        });
    }
}

template <class R>
__global__ void k_ccd_pg(Dev<R> D) {
    int qi = blockIdx.x * blockDim.x + threadIdx.x;
    if (qi >= D.nsv || !D.has_ground) return;
    int pv = D.sv[qi];
    d3 n = mk(D.gn[0], D.gn[1], D.gn[2]);
    d3 pp = mk((double)D.p[3 * pv], (double)D.p[3 * pv + 1], (double)D.p[3 * pv + 2]);
    double vn = dot(n, pp);
    if (!(vn < 0.0)) return;
    double d0 = dot(n, ld3(D.x + 3 * pv)) - D.goff;
    double a = fmin(1.0, (1.0 - D.ccd_shrink) * d0 / (-vn));
    if (!(a > 0.0)) a = 0.0;
    if (a < 1.0) {
        atomicMinPos(&D.alpha[D.grp0[pv]], a);
        atomicMinPos(&D.alpha_b[D.body[pv]], a);
    }
}

// ------------------------------------------------------ cached candidates
//
// Built at xref with margin delta: the stored boxes are inflated by
// infl = dhat + 2 delta, the query boxes are plain, so for positions y with
// max_v |y_v - xref_v| <= delta the list holds every pair with d(y) < dhat
// (proximity) and every pair whose swept boxes over a segment inside that
// ball overlap (CCD). The per-iteration kernels then apply the exact tests of
// the grid path to the listed pairs, giving the same contact and CCD
// candidate sets.

// append one int2 per calling thread with one atomic per warp
__device__ __forceinline__ void append_pair(int2* list, int* count, int cap, int a, int b) {
    unsigned m = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    int rank = __popc(m & ((1u << lane) - 1u));
    int base = cap;
    if (lane == leader && *(volatile int*)count < cap) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(m, base, leader);
    int k = base + rank;
    if (k < cap) list[k] = make_int2(a, b);
}

template <class R>
__global__ void k_cand_pt(Dev<R> D, const double* __restrict__ x) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int qi = (int)(gid / kSplitSwept), sub = (int)(gid % kSplitSwept);
    if (qi >= D.nsv) return;
    const int pv = D.sv[qi];
    float lo[3], hi[3];
    prim_box(D, &pv, 1, 4.f * D.xf[pv].w, lo, hi);
    grid_query<kSplitSwept>(D, lo, hi, D.nsf, sub, [&](int f) {
        if (pv == D.sf[3 * f] || pv == D.sf[3 * f + 1] || pv == D.sf[3 * f + 2]) return;
        append_pair(D.cand_pt, &D.cand_n[0], D.cand_cap, pv, f);
    });
}

template <class R>
__device__ __forceinline__ bool edges_adjacent(const Dev<R>& D, int i, int j) {
    int a0 = D.se[2 * i], a1 = D.se[2 * i + 1], b0 = D.se[2 * j], b1 = D.se[2 * j + 1];
    return a0 == b0 || a0 == b1 || a1 == b0 || a1 == b1;
}

template <class R>
__global__ void k_cand_ee(Dev<R> D, const double* __restrict__ x) {
    const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int i = (int)(gid / kSplitSwept), sub = (int)(gid % kSplitSwept);
    if (i >= D.nse) return;
    const int vid[2] = {D.se[2 * i], D.se[2 * i + 1]};
    float lo[3], hi[3];
    prim_box(D, vid, 2, 4.f * fmaxf(D.xf[vid[0]].w, D.xf[vid[1]].w), lo, hi);
    grid_query<kSplitSwept>(D, lo, hi, D.nse, sub, [&](int j) {
        if (j > i && !edges_adjacent(D, i, j)) append_pair(D.cand_ee, &D.cand_n[1], D.cand_cap, i, j);
    });
}

template <class R>
__global__ void k_set_cell_cand(Dev<R> D, double infl) {
    const double cs = fmax(D.cell, 2.0 * infl);
    *D.cellsz = cs;
    *D.cellinv = (float)(1.0 / cs);
}

// The list kernels take the cached candidate lists, or the pairs a grid
// query screened (one thread per pair either way).
template <class R>
__global__ void k_prox_pt_list(Dev<R> D, const double* __restrict__ x, ContactBuf C, const int2* list, const int* cnt,
                               int cap,
                              const int* skip) {
    if (skip && *skip) return;  // the fused query handles an overflowed list
    int n = min(*cnt, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int2 q = list[k];
        pt_try(D, x, C, q.x, q.y);
    }
}

template <class R>
__global__ void k_prox_ee_list(Dev<R> D, const double* __restrict__ x, ContactBuf C, const int2* list, const int* cnt,
                               int cap,
                              const int* skip) {
    if (skip && *skip) return;  // the fused query handles an overflowed list
    int n = min(*cnt, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int2 q = list[k];
        ee_try(D, x, C, q.x, q.y);
    }
}

// Screening passes over a cached candidate list: the proximity pairs that
// need the FP64 distance (FP32 lower bound below dhat) and the CCD pairs that
// need the FP64 walk are appended to the scratch list gpair, which the list
// kernels below then finish one thread per pair with all lanes of a warp on
// the FP64 path (FP64 runs at a small fraction of the FP32 rate here, and a
// warp that mixes screened-out pairs with one FP64 pair issues the FP64 code
// for that one lane). A pair that does not fit the scratch list is finished
// in the screening pass itself, so each pair is handled exactly once.
template <class R, int kKind>
__global__ void __launch_bounds__(kT, 8) k_prox_screen(Dev<R> D, const double* __restrict__ x, ContactBuf C, const int2* list,
                              const int* cnt, int cap) {
    const int n = min(*cnt, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int2 q = list[k];
        const bool need = kKind == 0 ? pt_needed(D, q.x, q.y) : ee_needed(D, q.x, q.y);
        if (need && !append_ok(D.gpair, D.gpair_n, D.gpair_cap, q.x, q.y)) {
            if (kKind == 0)
                pt_try(D, x, C, q.x, q.y);
            else
                ee_try(D, x, C, q.x, q.y);
        }
    }
}

template <class R, int kKind>
__global__ void __launch_bounds__(kT, 6) k_ccd_screen(Dev<R> D, const int2* list, const int* cnt, int cap) {
    const int n = min(*cnt, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int2 q = list[k];
        int v[4];
        float lo[3], hi[3], blo[3], bhi[3];
        if (kKind == 0) {
            v[0] = q.x;
            v[1] = D.sf[3 * q.y];
            v[2] = D.sf[3 * q.y + 1];
            v[3] = D.sf[3 * q.y + 2];
            prim_box(D, v, 1, 0.f, lo, hi);
            prim_box(D, v + 1, 3, 0.f, blo, bhi);
        } else {
            v[0] = D.se[2 * q.x];
            v[1] = D.se[2 * q.x + 1];
            v[2] = D.se[2 * q.y];
            v[3] = D.se[2 * q.y + 1];
            prim_box(D, v, 2, 0.f, lo, hi);
            prim_box(D, v + 2, 2, 0.f, blo, bhi);
        }
        if (overlap(lo, hi, blo, bhi)) ccd_pair(D, kKind, v, &q);
    }
}

template <class R>
__global__ void k_ccd_pt_list(Dev<R> D, const int2* list, const int* cnt, int cap,
                              const int* skip) {
    if (skip && *skip) return;  // the fused query handles an overflowed list
    int n = min(*cnt, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int2 q = list[k];
        int v[4] = {q.x, D.sf[3 * q.y], D.sf[3 * q.y + 1], D.sf[3 * q.y + 2]};
        float lo[3], hi[3], tlo[3], thi[3];
        prim_box(D, v, 1, 0.f, lo, hi);
        prim_box(D, v + 1, 3, 0.f, tlo, thi);
        if (overlap(lo, hi, tlo, thi)) ccd_pair(D, 0, v);
    }
}

template <class R>
__global__ void k_ccd_ee_list(Dev<R> D, const int2* list, const int* cnt, int cap,
                              const int* skip) {
    if (skip && *skip) return;  // the fused query handles an overflowed list
    int n = min(*cnt, cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int2 q = list[k];
        int v[4] = {D.se[2 * q.x], D.se[2 * q.x + 1], D.se[2 * q.y], D.se[2 * q.y + 1]};
        float lo[3], hi[3], blo[3], bhi[3];
        prim_box(D, v, 2, 0.f, lo, hi);
        prim_box(D, v + 2, 2, 0.f, blo, bhi);
        if (overlap(lo, hi, blo, bhi)) ccd_pair(D, 1, v);
    }
}

// global-step ablation: every subdomain and body takes the smallest step
// bound (alpha_min after verification), and the line search's tiers see no
// per-subdomain or per-body spread
template <class R>
__global__ void k_global_alpha(Dev<R> D) {
    const double a = D.S->alpha_min;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < D.ngroups[0]; g += gridDim.x * blockDim.x) D.alpha[g] = a;
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < D.nbody; b += gridDim.x * blockDim.x) D.alpha_b[b] = a;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        D.S->alpha_max = a;
        D.S->alpha_bmin = a;
        D.S->alpha_bmax = a;
    }
}

template <class R>
__global__ void k_fill(Dev<R> D, double* a, int n, double v) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

template <class R>
__global__ void k_ccd_begin(Dev<R> D) {
    Scalars* S = D.S;
    S->n_straddle = 0;
    S->overflow &= ~2;
    for (int i = 0; i < 3 * kCcdPasses; ++i) D.vflags[i] = 0;
    S->ccd_viol = S->ccd_viol_b = 0;
    S->ccd_uniform = S->ccd_uniform_b = 0;
    S->ccd_passes = S->ccd_passes_b = 0;
}

// One grouping of the vertices (level-0 subdomains or bodies) with its step
// sizes, verification scratch and status words.
struct Grouping {
    const int* of;        // group of each vertex
    double* alpha;
    double* shrink;       // scratch, n
    double* third;        // scratch, n
    double* fourth;       // scratch, n
    int n;
    int* viol;
    int* state;           // 0 running, 1 uniform fallback, 2 verified
    int* passes;
    double* amin;         // minimum before verification (the uniform step); on exit the final minimum
    double* amax;         // on exit the final maximum
    double* fmin;         // scratch scalars for the final minimum and maximum
    double* fmax;
};

// does straddling pair k need the FP64 walk under grouping G's steps a?
// False where it cannot be violated: all four vertices in one group, one
// common step, or FP32 bounds that prove rho = 1. prev: the steps of the
// previous pass (nullptr in the first): a pair none of whose groups changed
// since moves exactly as it did when it was last checked, and then it was
// not violated (a violation lowers at least one of its groups), so it is not
// checked again
template <class R>
__device__ __forceinline__ bool pair_needs_walk(const Dev<R>& D, const Grouping& G, const double* a,
                                                const double* prev, int k, int v[4]) {
    const int4 q = D.str_v[k];
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
    const int g0 = G.of[v[0]];
    if (G.of[v[1]] == g0 && G.of[v[2]] == g0 && G.of[v[3]] == g0) return false;
    if (prev) {
        bool same = true;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gj = G.of[v[j]];
            same = same && a[gj] == prev[gj];
        }
        if (same) return false;
    }
    // groups with one common step a move the pair uniformly by a p, and each
    // group's a is at most this pair's own safe fraction (the minimum over
    // the pairs touching it, this one included): safe
    {
        const double a0 = a[g0];
        if (a[G.of[v[1]]] == a0 && a[G.of[v[2]]] == a0 && a[G.of[v[3]]] == a0) return false;
    }
    const int kind = D.str_t[k];
    {
        // the FP64 walk returns exactly 1 where the FP32 distance bound
        // exceeds the largest relative displacement of the actual motion
        // (CUBICSAFE starts at alpha_l >= 1): skip it there
        float P[4][3], pm = 0.f;
        for (int j = 0; j < 4; ++j) {
            const float sj = (float)a[G.of[v[j]]];
            const R* qq = D.p + 3 * v[j];
            P[j][0] = sj * (float)qq[0];
            P[j][1] = sj * (float)qq[1];
            P[j][2] = sj * (float)qq[2];
            pm = fmaxf(pm, sqrtf(P[j][0] * P[j][0] + P[j][1] * P[j][1] + P[j][2] * P[j][2]));
        }
        float lr = 0.f;
        for (int i = 0; i < (kind == 0 ? 1 : 2); ++i)
            for (int j = (kind == 0 ? 1 : 2); j < 4; ++j) {
                const float dx = P[i][0] - P[j][0], dy = P[i][1] - P[j][1], dz = P[i][2] - P[j][2];
                lr = fmaxf(lr, sqrtf(dx * dx + dy * dy + dz * dz));
            }
        const float lim = pair_dist_lb(D, kind, v) * (1.f - (float)D.ccd_shrink);
        if (lim > 1.001f * lr + 2e-3f * pm) return false;
    }
    return true;
}

// the FP64 walk of straddling pair k (vertices v) with the actual motion:
// violated when it cannot take the whole step; then m = the smallest step of
// the groups it touches
template <class R>
__device__ __forceinline__ bool pair_walk_violated(const Dev<R>& D, const Grouping& G, const double* a, int k,
                                                   const int v[4], double& m) {
    const double rho = pair_alpha(D, D.str_t[k], v, D.x, D.p, a, G.of);
    if (!(rho < 1.0)) return false;
    m = a[G.of[v[0]]];
    for (int j = 1; j < 4; ++j) m = fmin(m, a[G.of[v[j]]]);
    return true;
}

// Verification of the straddling candidates for both groupings (level-0
// subdomains and bodies, side by side) in one cooperative launch: per pass,
// every straddling pair is re-checked with the actual motion alpha_g(v) p_v;
// a violating pair lowers every group it touches to the pair's smallest alpha
// (the pair then moves uniformly on a segment already checked). A grouping
// stops at its first clean pass; after kCcdPasses passes with a violation, or
// when the candidate list overflowed, it takes the uniform step
// min_g alpha_g. A pass reads the steps from buffer k mod 4 and takes minima
// into buffer k + 1 mod 4 (each group's own step and the violations' minima,
// both commutative), reads the previous pass's steps from buffer k + 3 mod 4
// (pairs whose groups all kept their step are not checked again), while
// buffer k + 2 mod 4, which nothing touches in this pass, is reset for the
// next. It has two grid barriers: the first after the FP32 screen of every
// pair, which collects the pairs that need the FP64 walk into a compact list
// (the scratch pair list, free at this point), the second after the walks of
// that list, so that the lanes of a warp walk together instead of one lane
// at a time.
// Grid-wide barriers are cooperative-groups syncs of a co-resident grid
// (cudaLaunchCooperativeKernel); every thread executes the same sequence.
template <class R>
__global__ void __launch_bounds__(256, 2) k_verify_all(Dev<R> D, Grouping G0, Grouping G1) {
    cg::grid_group grid = cg::this_grid();
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int nstr = min(D.S->n_straddle, D.straddle_cap);
    const bool overflow = (D.S->overflow & 2) != 0;
    const Grouping* Gs[2] = {&G0, &G1};
    int* vcnt = D.vflags + 2 * kCcdPasses;  // compact-list length of each pass (zeroed by k_ccd_begin)
    if (tid == 0) {
        *G0.amin = *G1.amin = 1.0;
        *G0.fmin = *G1.fmin = 1.0;
        *G0.fmax = *G1.fmax = 0.0;
    }
    grid.sync();
    for (int gi = 0; gi < 2; ++gi) {
        const Grouping& G = *Gs[gi];
        double mn = 1.0;
        for (int g = tid; g < G.n; g += nth) {
            mn = fmin(mn, G.alpha[g]);
            G.shrink[g] = 1.0;  // the target of pass 0
        }
        for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        if (lane == 0 && mn < 1.0) atomicMinPos(G.amin, mn);
    }
    grid.sync();
    // state 0 running, 1 uniform fallback, 2 verified; fin = the buffer
    // holding a verified grouping's steps
    int state[2] = {overflow ? 1 : 0, overflow ? 1 : 0};
    int passes[2] = {overflow ? -1 : 0, overflow ? -1 : 0};
    int fin[2] = {0, 0};
    for (int pass = 0; pass < kCcdPasses && (state[0] == 0 || state[1] == 0); ++pass) {
        for (int gi = 0; gi < 2; ++gi) {
            if (state[gi] != 0) continue;
            const Grouping& G = *Gs[gi];
            double* bufs[4] = {G.alpha, G.shrink, G.third, G.fourth};
            const double* A = bufs[pass % 4];
            double* B = bufs[(pass + 1) % 4];
            double* Z = bufs[(pass + 2) % 4];
            const double* Pv = pass > 0 ? bufs[(pass + 3) % 4] : nullptr;
            int* vf = D.vflags + gi * kCcdPasses;
            for (int g = tid; g < G.n; g += nth) {
                atomicMinPos(&B[g], A[g]);
                Z[g] = 1.0;
            }
            for (int k = tid; k < nstr; k += nth) {
                int v[4];
                double m;
                // pairs that need the FP64 walk go to the compact list of this
                // pass; one that does not fit is walked here
                if (pair_needs_walk(D, G, A, Pv, k, v) &&
                    !append_ok(D.gpair, vcnt + pass, D.gpair_cap, k, gi) && pair_walk_violated(D, G, A, k, v, m)) {
                    vf[pass] = 1;
                    for (int j = 0; j < 4; ++j) atomicMinPos(&B[G.of[v[j]]], m);
                }
            }
        }
        grid.sync();
        // the walks of the compact list, every lane of a warp on one
        {
            const int nw = min(__ldcg(vcnt + pass), D.gpair_cap);
            for (int e = tid; e < nw; e += nth) {
                const int2 q = __ldcg(&D.gpair[e]);
                const int k = q.x, gi = q.y;
                const Grouping& G = *Gs[gi];
                double* bufs[4] = {G.alpha, G.shrink, G.third, G.fourth};
                const double* A = bufs[pass % 4];
                double* B = bufs[(pass + 1) % 4];
                const int4 qv = D.str_v[k];
                const int v[4] = {qv.x, qv.y, qv.z, qv.w};
                double m;
                if (pair_walk_violated(D, G, A, k, v, m)) {
                    D.vflags[gi * kCcdPasses + pass] = 1;
                    for (int j = 0; j < 4; ++j) atomicMinPos(&B[G.of[v[j]]], m);
                }
            }
        }
        grid.sync();
        for (int gi = 0; gi < 2; ++gi) {
            if (state[gi] != 0) continue;
            if (__ldcg(&D.vflags[gi * kCcdPasses + pass]) == 0) {
                state[gi] = 2;
                passes[gi] = pass + 1;
                fin[gi] = pass % 4;
            }
        }
    }
    // write the result into alpha (the verified buffer, or the uniform step),
    // gathering its minimum and maximum on the way
    for (int gi = 0; gi < 2; ++gi) {
        const Grouping& G = *Gs[gi];
        if (state[gi] == 0) {
            state[gi] = 1;
            passes[gi] = -1;
        }
        const double* src = fin[gi] == 0 ? G.alpha : fin[gi] == 1 ? G.shrink : fin[gi] == 2 ? G.third : G.fourth;
        const double a_uni = __ldcg(G.amin);
        double lo = 1.0, hi = 0.0;
        for (int g = tid; g < G.n; g += nth) {
            const double a = state[gi] == 1 ? a_uni : src[g];
            if (state[gi] == 1 || fin[gi] != 0) G.alpha[g] = a;
            lo = fmin(lo, a);
            hi = fmax(hi, a);
        }
        for (int o = 16; o > 0; o >>= 1) {
            lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            if (lo < 1.0) atomicMinPos(G.fmin, lo);
            if (hi > 0.0) atomicMaxPos(G.fmax, hi);
        }
    }
    grid.sync();
    if (tid == 0) {
        for (int gi = 0; gi < 2; ++gi) {
            const Grouping& G = *Gs[gi];
            *G.state = state[gi];
            *G.passes = passes[gi];
            *G.viol = state[gi] != 2;
            *G.amin = *G.fmin;
            *G.amax = *G.fmax;
        }
    }
}

// Cooperative launches of all scenes in the process are ordered on the GPU:
// each one's stream first waits for the previous one (an event recorded after
// it, on whatever stream it ran), so two grids that need all their blocks
// resident at once never wait on each other's blocks when several scenes step
// concurrently (ipc_server). Other kernels still overlap freely.
std::mutex g_coop_mu;

template <class R>
void verify_groupings(const Dev<R>& D, const Grouping& sub, const Grouping& bod, cudaStream_t st) {
    static const int nblocks = [] {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_verify_all<R>, 256, 0);
        int n = sms * (per < 2 ? per : 2);
        return n < 1 ? 1 : n;
    }();
    static cudaEvent_t last = [] {
        cudaEvent_t e = nullptr;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        return e;
    }();
    Dev<R> Dc = D;
    Grouping a = sub, b = bod;
    void* args[] = {&Dc, &a, &b};
    std::lock_guard<std::mutex> lock(g_coop_mu);
    if (last) cudaStreamWaitEvent(st, last, 0);
    KL(cudaLaunchCooperativeKernel((const void*)k_verify_all<R>, dim3(nblocks), dim3(256), args, 0, st));
    if (last) cudaEventRecord(last, st);
}

}  // namespace

template <class R>
void launch_detect(const Dev<R>& D, const double* x, const ContactBuf& C, cudaStream_t st) {
    KL(k_reset_detect<R><<<1, 1, 0, st>>>(D, C));
    if (D.nsv) KL(k_vert_f32<R><<<nblk(D.nsv), kT, 0, st>>>(D, x, (const R*)nullptr));
    int* gin = D.gin;
    const float dh = round_up_f(D.dhat);
    build_grid<R>(D, D.sf, 3, D.nsf, dh, gin, false, st);
    cudaMemsetAsync(D.gpair_n, 0, 2 * sizeof(int), st);
    if (D.nsv) {
        KL(k_prox_pt<R, false><<<nblk((long long)D.nsv * kSplitProx), kT, 0, st>>>(D, x, C));
        KL(k_prox_pt_list<R><<<1184, kT, 0, st>>>(D, x, C, D.gpair, D.gpair_n, D.gpair_cap, D.gpair_n + 1));
        KL(k_prox_pt<R, true><<<1184, kT, 0, st>>>(D, x, C));
    }
    build_grid<R>(D, D.se, 2, D.nse, dh, gin, false, st);
    cudaMemsetAsync(D.gpair_n, 0, 2 * sizeof(int), st);
    if (D.nse) {
        KL(k_prox_ee<R, false><<<nblk((long long)D.nse * kSplitProx), kT, 0, st>>>(D, x, C));
        KL(k_prox_ee_list<R><<<1184, kT, 0, st>>>(D, x, C, D.gpair, D.gpair_n, D.gpair_cap, D.gpair_n + 1));
        KL(k_prox_ee<R, true><<<1184, kT, 0, st>>>(D, x, C));
    }
    if (D.nsv) KL(k_prox_pg<R><<<nblk(D.nsv), kT, 0, st>>>(D, x, C));
}

template <class R>
void launch_ccd(const Dev<R>& D, cudaStream_t st) {
    int ng = D.ngroups[0];
    KL(k_ccd_begin<R><<<1, 1, 0, st>>>(D));
    KL(k_fill<R><<<nblk(ng), kT, 0, st>>>(D, D.alpha, ng, 1.0));
    KL(k_fill<R><<<nblk(D.nbody), kT, 0, st>>>(D, D.alpha_b, D.nbody, 1.0));
    if (D.nsv) KL(k_vert_f32<R><<<nblk(D.nsv), kT, 0, st>>>(D, D.x, (const R*)D.p));
    int* gin = D.gin;
    build_grid<R>(D, D.sf, 3, D.nsf, 0.f, gin, true, st);
    cudaMemsetAsync(D.gpair_n, 0, 2 * sizeof(int), st);
    if (D.nsv) {
        KL(k_ccd_pt<R, false><<<nblk((long long)D.nsv * kSplitSwept), kT, 0, st>>>(D));
        KL(k_ccd_pt_list<R><<<1184, kT, 0, st>>>(D, D.gpair, D.gpair_n, D.gpair_cap, D.gpair_n + 1));
        KL(k_ccd_pt<R, true><<<1184, kT, 0, st>>>(D));
    }
    build_grid<R>(D, D.se, 2, D.nse, 0.f, gin, true, st);
    cudaMemsetAsync(D.gpair_n, 0, 2 * sizeof(int), st);
    if (D.nse) {
        KL(k_ccd_ee<R, false><<<nblk((long long)D.nse * kSplitSwept), kT, 0, st>>>(D));
        KL(k_ccd_ee_list<R><<<1184, kT, 0, st>>>(D, D.gpair, D.gpair_n, D.gpair_cap, D.gpair_n + 1));
        KL(k_ccd_ee<R, true><<<1184, kT, 0, st>>>(D));
    }
    if (D.nsv) KL(k_ccd_pg<R><<<nblk(D.nsv), kT, 0, st>>>(D));
    Scalars* S = D.S;
    Grouping sub{D.grp0, D.alpha, D.shrink, D.shrink3, D.shrink4, ng, &S->ccd_viol, &S->ccd_uniform, &S->ccd_passes,
                 &S->alpha_min, &S->alpha_max, &S->vstat[0], &S->vstat[1]};
    Grouping bod{D.body, D.alpha_b, D.shrink_b, D.shrink3_b, D.shrink4_b, D.nbody, &S->ccd_viol_b, &S->ccd_uniform_b,
                 &S->ccd_passes_b, &S->alpha_bmin, &S->alpha_bmax, &S->vstat[2], &S->vstat[3]};
    verify_groupings(D, sub, bod, st);
}

template <class R>
void launch_cand_build(const Dev<R>& D, const double* x, double delta, cudaStream_t st) {
    const double infl = D.dhat + 2.001 * delta;
    cudaMemsetAsync(D.cand_n, 0, 2 * sizeof(int), st);
    if (D.nsv) KL(k_vert_f32<R><<<nblk(D.nsv), kT, 0, st>>>(D, x, (const R*)nullptr));
    int* gin = D.gin;
    for (int pass = 0; pass < 2; ++pass) {
        const int* prims = pass == 0 ? D.sf : D.se;
        int nper = pass == 0 ? 3 : 2, nprim = pass == 0 ? D.nsf : D.nse;
        cudaMemsetAsync(D.gcount, 0, sizeof(int) * (D.nbuckets + 1), st);
        cudaMemsetAsync(D.gfill, 0, sizeof(int) * D.nbuckets, st);
        cudaMemsetAsync(D.gtotal, 0, sizeof(int), st);
        cudaMemsetAsync(D.gnlarge, 0, sizeof(int), st);
        KL(k_set_cell_cand<R><<<1, 1, 0, st>>>(D, infl));
        if (nprim > 0) KL(k_grid_count<R><<<nblk(nprim), kT, 0, st>>>(D, prims, nper, nprim, round_up_f(infl), gin));
        scan_exclusive(D.gcount, D.gstart, D.nbuckets, D.gtmp, st);
        if (nprim > 0) KL(k_grid_fill<R><<<nblk(nprim), kT, 0, st>>>(D, nprim, gin));
        if (pass == 0 && D.nsv) KL(k_cand_pt<R><<<nblk((long long)D.nsv * kSplitSwept), kT, 0, st>>>(D, x));
        if (pass == 1 && D.nse) KL(k_cand_ee<R><<<nblk((long long)D.nse * kSplitSwept), kT, 0, st>>>(D, x));
    }
    cudaMemcpyAsync(D.xref, x, sizeof(double) * 3 * (size_t)D.nv, cudaMemcpyDeviceToDevice, st);
}

template <class R>
void launch_detect_list(const Dev<R>& D, const double* x, const ContactBuf& C, cudaStream_t st) {
    KL(k_reset_detect<R><<<1, 1, 0, st>>>(D, C));
    if (D.nsv) KL(k_vert_f32<R><<<nblk(D.nsv), kT, 0, st>>>(D, x, (const R*)nullptr));
    // FP32 screen of each cached list into the scratch list, then the FP64
    // tests of the screened pairs
    cudaMemsetAsync(D.gpair_n, 0, 2 * sizeof(int), st);
    KL(k_prox_screen<R, 0><<<1184, kT, 0, st>>>(D, x, C, D.cand_pt, &D.cand_n[0], D.cand_cap));
    KL(k_prox_pt_list<R><<<1184, kT, 0, st>>>(D, x, C, D.gpair, D.gpair_n, D.gpair_cap, nullptr));
    cudaMemsetAsync(D.gpair_n, 0, 2 * sizeof(int), st);
    KL(k_prox_screen<R, 1><<<1184, kT, 0, st>>>(D, x, C, D.cand_ee, &D.cand_n[1], D.cand_cap));
    KL(k_prox_ee_list<R><<<1184, kT, 0, st>>>(D, x, C, D.gpair, D.gpair_n, D.gpair_cap, nullptr));
    if (D.nsv) KL(k_prox_pg<R><<<nblk(D.nsv), kT, 0, st>>>(D, x, C));
}

template <class R>
void launch_ccd_list(const Dev<R>& D, cudaStream_t st, int part) {
    int ng = D.ngroups[0];
    if (part != 2) {  // per-pair bounds (capturable in a graph)
        KL(k_ccd_begin<R><<<1, 1, 0, st>>>(D));
        KL(k_fill<R><<<nblk(ng), kT, 0, st>>>(D, D.alpha, ng, 1.0));
        KL(k_fill<R><<<nblk(D.nbody), kT, 0, st>>>(D, D.alpha_b, D.nbody, 1.0));
        if (D.nsv) KL(k_vert_f32<R><<<nblk(D.nsv), kT, 0, st>>>(D, D.x, (const R*)D.p));
        // FP32 screen of each cached list (pairs that need the FP64 walk into
        // the scratch list), then the walks of the screened pairs
        cudaMemsetAsync(D.gpair_n, 0, 2 * sizeof(int), st);
        KL(k_ccd_screen<R, 0><<<1184, kT, 0, st>>>(D, D.cand_pt, &D.cand_n[0], D.cand_cap));
        KL(k_ccd_pt_list<R><<<1184, kT, 0, st>>>(D, D.gpair, D.gpair_n, D.gpair_cap, nullptr));
        cudaMemsetAsync(D.gpair_n, 0, 2 * sizeof(int), st);
        KL(k_ccd_screen<R, 1><<<1184, kT, 0, st>>>(D, D.cand_ee, &D.cand_n[1], D.cand_cap));
        KL(k_ccd_ee_list<R><<<1184, kT, 0, st>>>(D, D.gpair, D.gpair_n, D.gpair_cap, nullptr));
        if (D.nsv) KL(k_ccd_pg<R><<<nblk(D.nsv), kT, 0, st>>>(D));
    }
    if (part != 1) {  // verification: one cooperative launch, ordered across scenes
        Scalars* S = D.S;
        Grouping sub{D.grp0, D.alpha, D.shrink, D.shrink3, D.shrink4, ng, &S->ccd_viol, &S->ccd_uniform, &S->ccd_passes,
                     &S->alpha_min, &S->alpha_max, &S->vstat[0], &S->vstat[1]};
        Grouping bod{D.body, D.alpha_b, D.shrink_b, D.shrink3_b, D.shrink4_b, D.nbody, &S->ccd_viol_b, &S->ccd_uniform_b,
                     &S->ccd_passes_b, &S->alpha_bmin, &S->alpha_bmax, &S->vstat[2], &S->vstat[3]};
        verify_groupings(D, sub, bod, st);
    }
}

template <class R>
void launch_global_alpha(const Dev<R>& D, cudaStream_t st) {
    KL(k_global_alpha<R><<<nblk(std::max(D.ngroups[0], D.nbody)), kT, 0, st>>>(D));
}

#define INST(R)                                                                               \
    template void launch_detect<R>(const Dev<R>&, const double*, const ContactBuf&, cudaStream_t); \
    template void launch_ccd<R>(const Dev<R>&, cudaStream_t);                                  \
    template void launch_cand_build<R>(const Dev<R>&, const double*, double, cudaStream_t);    \
    template void launch_detect_list<R>(const Dev<R>&, const double*, const ContactBuf&, cudaStream_t); \
    template void launch_ccd_list<R>(const Dev<R>&, cudaStream_t, int);          \
    template void launch_global_alpha<R>(const Dev<R>&, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace ipcb
