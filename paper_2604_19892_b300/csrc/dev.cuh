// Device-side view of one scene and shared device helpers.
//
// Layout in HBM (one scene; R = double in FP64 mode, float in FP32 mode):
//   vertices   x, x~, x_start, x_try, v: double[3 nv] (AoS xyz); g, g_try,
//              z, z_prev, p: R[3 nv]; mass: R[nv]
//   tets       int4 tets[nt]; rest inverse B and the projected elastic
//              Hessian h^2 V dP/dF (45 packed symmetric entries) in 32-tet
//              packets [nt/32][n][32] so a warp reads 128-byte lines
//   contacts   structure of arrays, capacity cap, two buffers (current and
//              trial) swapped on an accepted step, plus the restart snapshot
//              C_base with an open-addressing key table
//   MAS        all levels' 96x96 inverses B = W'^T W' as their lower
//              triangular factors W' packed by columns, R[nblocks][4656]
//              (level 0 first); blocks assembled in double
//   CCD        alpha per level-0 subdomain (double) and the straddling
//              candidate list for the verification passes
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "host_mesh.h"

namespace ipcb {

// Every kernel launch of the library goes through KL(...), which counts it.
void count_launch();
#define KL(...) (::ipcb::count_launch(), __VA_ARGS__)

constexpr int kMaxK = 16;          // Woodbury vectors per subdomain
constexpr int kPack = 32;          // tets per packet
constexpr int kH = 45;             // packed symmetric 9x9
// A subdomain block's inverse is kept as its factor W' (B = W'^T W', W'
// lower triangular), packed by columns with 4-row alignment: column j = 4a + b
// holds rows 4a..95 (the rows 4a..j-1 above the diagonal are zero) starting
// at wcol(j), a multiple of 4, so 16-byte vector loads of 4 rows stay
// aligned. 4,800 values per block (the plain triangle has 4,656).
constexpr int kW = 4800;
// BF16 factor storage (IPC_PREC_BF16_MAS): W' as its 21 lower 16 x 16 tiles,
// tile (i, j), i >= j, at index i (i + 1) / 2 + j, each row-major (the
// upper half of a diagonal tile is zero): 5,376 values, 10,752 bytes
constexpr int kT16 = 16;
constexpr int kNT16 = kBlk / kT16;
constexpr int kW16 = kNT16 * (kNT16 + 1) / 2 * kT16 * kT16;
__host__ __device__ __forceinline__ int wcol(int j) {
    const int a = j >> 2, b = j & 3;
    return 4 * (kBlk * a - 2 * a * (a - 1)) + b * (kBlk - 4 * a);
}

// Per-scene scalars living in device memory; the host reads them once per
// energy-check trial.
struct Scalars {
    // reductions of the current iteration
    double gz, gp, gzprev;         // g.z, g.p_k, g.z_k
    double zHz, zHp, pHp;          // quadratic forms of H~ (Eq. 13-15)
    double znorm;                  // max_v |z_v| (as double bits, atomicMax)
    double pmax;                   // max_v |p_v|
    double maxdisp;                // max_v |x_v - xref_v|
    double mu, nu;
    // energies
    double E_k, E_try;
    double min_dist;               // of the trial contact set
    int restart;
    int accepted;
    int ccd_viol;                  // verification found a violation
    int ccd_uniform;               // 2 verified, 1 fell back to uniform alpha
    int ccd_passes;                // verification passes run
    int ccd_viol_b, ccd_uniform_b, ccd_passes_b;  // the same for the body grouping
    double alpha_bmin, alpha_bmax; // smallest / largest per-body step
    double vstat[4];               // verification scratch: final min / max per grouping
    int n_upd;                     // classified updates
    int n_straddle;                // straddling CCD candidates
    int overflow;                  // bit flags: 1 contacts, 2 straddle, 4 upd
    int nan_flag;
    int async_timeout;             // a bounded wait on an asynchronous copy ran out
    int nonpos;                    // a contact of the last detection has d <= 0
    // first block apply with a non-finite result: block, updates used,
    // max |rhs| (g and U columns), max |Y|, max |lambda|, max dS
    int dbg_block, dbg_ns;
    double dbg_rhs, dbg_y, dbg_lam, dbg_ds;
    double alpha_min, alpha_max;
    double beta;                   // uniform step of the current trial (0 = per-subdomain)
};

struct ContactBuf {
    int* count;                    // device scalar
    int* type;
    int4* v;
    unsigned long long* key;
    double* d;
    double* k;                     // kappa b''(d)
    double* bp;                    // kappa b'(d)
    double* r;                     // 3 per contact: unit direction (p - c)/d or plane normal
    double* w;                     // 4 per contact: grad d = (w_j r) per vertex
};

// four values of one vertex vector, one aligned 16-byte (FP32) load
template <class R>
struct alignas(4 * sizeof(R)) V4 {
    R x, y, z, w;
};

template <class R>
struct Dev {
    // sizes
    int nv, nt, nsv, nsf, nse, nlev, ntp;   // ntp = number of 32-tet packets
    int ngroups[kMaxLevels], nnodes[kMaxLevels], blk_off[kMaxLevels + 1];
    int cap;                               // contact capacity
    int upd_cap, straddle_cap;
    // parameters
    double h, dhat, kappa, eps_conv, delta, cos_rot, ccd_shrink, eps_sing, eps_abs;
    int K, ls_max;
    // energy check: accept E_try <= E_k + tau_rel |E_k| + tau_abs (rounding
    // allowance of the two computed energies)
    double tau_rel, tau_abs;
    int wait_polls;                        // polls of a bounded wait on a bulk copy
    int apply_ctas;                        // persistent plain block apply: CTAs per SM (autotuned; 0 = default)
    double gravity[3];
    int has_ground;
    double gn[3], goff;
    double cell;                           // broad-phase base cell size
    // mesh
    const int4* tets;
    const R* tetB;                         // [ntp][9][32] rest inverse (row-major 3x3)
    const double* tet_vol;                 // V
    const double* tet_mu;
    const double* tet_lam;
    float piv32;                           // FP32 inversion: pivot floor that sends a block to FP64
    const float2* tet_ec;                  // FP32 bulk: [nt][3] h^2 V mu / 2, h^2 V mu, h^2 V lam / 2 as float hi, lo
    const R* mass;
    const double* massd;
    const int* sv;
    const int* sf;                         // 3 per surface tri
    const int* se;                         // 2 per surface edge
    // hierarchy
    const int* node_of_vert[kMaxLevels];   // l >= 1: level-l node of each vertex (l = 0: grp0 unused)
    const int* grp0;                       // level-0 group of each vertex
    const int* slot0;
    const int* members[kMaxLevels];        // per level: ngroups*32 node ids (-1 pad)
    const int* grp_of_node[kMaxLevels];
    const int* slot_of_node[kMaxLevels];
    // state
    double *x, *xt, *xs, *xtry, *v;
    R *g, *gtry, *z, *zprev, *p;
    R* zp4;                                // [nv][2][4]: z and p packed for the forms gathers
    R* hess;                               // [ntp][45][32]
    R* blocks;                             // nblocks * kW: packed factors W' (B = W'^T W')
    void* blocks16;                        // BF16 factors (nblocks * kW16 bf16), or null: FP32 / FP64 factors in blocks
    R* jac;                                // 3x3 block-Jacobi preconditioner (mas_mode 3): nv x 9, else null
    double* asmb;                          // level-0 assembly buffer (FP64)
    double* asmbc;                         // coarse-level assembly buffer (FP64)
    const double* mdiag;                   // per block: mass diagonal (96 entries), fixed
    int ncon, nitem;                       // coarse elastic assembly: contributions, summation items
    R* cval;                               // 12 x ncon: 3x3 value of each contribution (+3 pad)
    const int* tcon_off;                   // per tet (nt + 1): its contributions,
    const int2* tcon;                      //   (slot in cval, vertex masks: bits 0-3 set i, 4-7 set j)
    const int4* item;                      // nitem + 1: global block, slot i, slot j | split << 8, first entry
    int* invflag;                          // level-0 blocks to re-invert in FP64
    int* pivfix;                           // blocks whose final factorisation floored or raised a pivot (last restart)
    R* coarse_r;                           // restricted residuals, 3 * nnodes[l] per level, offsets coarse_off
    R* coarse_y;
    int coarse_off[kMaxLevels + 1];
    // contacts
    ContactBuf C, Ct, Cb;                  // current, trial, base (restart snapshot)
    unsigned long long* bkeys;             // base key table, size btab (power of 2)
    int* bidx;
    int btab;
    // updates (classified contacts with dS > 0)
    int* upd_c;                            // contact index into C
    double* upd_dS;
    int* upd_cnt;                          // per level-0 group: number of touching updates
    int* upd_off;                          // exclusive scan, ngroups0 + 1
    int* upd_cur;                          // fill cursors
    int* upd_list;                         // update indices grouped by subdomain
    int* topk;                             // ngroups0 * K update ids (-1 empty)
    // CCD
    double* alpha;                         // per level-0 group
    double* shrink;
    double* shrink3;                       // second verification scratch per level-0 subdomain
    double* shrink4;                       // third verification scratch per level-0 subdomain
    double* pg_k;                          // per coarse node (offset coarse_off[l] / 3): the summed
                                           // stiffness of its point-ground contacts (RebuildMAS scratch)
    int nbody;
    const int* body;                       // connected body of each vertex
    double* alpha_b;                       // per body
    double* shrink_b;
    double* shrink3_b;
    double* shrink4_b;
    int* vflags;                           // verification: violation flag per grouping and pass
    int4* str_v;                           // straddling candidates: vertices
    int* str_t;                            // 0 PT (p, t0, t1, t2), 1 EE (a0, a1, b0, b1)
    // broad-phase grid (shared by proximity and CCD queries)
    int nbuckets;                          // power of 2
    int gcap;                              // entry capacity
    int* gcount;                           // bucket counts (nbuckets + 1)
    int* gstart;                           // bucket starts (nbuckets + 1)
    int* gfill;                            // fill cursor per bucket
    float4* gbox;                          // per entry: FP32 box lo (.w: primitive id bits), hi
    unsigned long long* gcell;             // packed cell of each entry
    int* gtotal;                           // scalar: entries used
    int* glarge;                           // primitives too large for the grid
    int* gnlarge;
    int* gin;                              // per stored primitive: 1 if binned
    int* gtmp;                             // scan temporaries
    float4* pbox;                          // per stored primitive: FP32 lo, hi (grown by the error bounds)
    float4* xf;                            // FP32 surface positions at the evaluation point (.w: error bound)
    float4* xpf;                           // FP32 surface positions at x + p (CCD), else a copy of xf
    float4* xsplit;                        // 2 nv: FP32 hi and lo parts of the energy point (FP32 bulk)
    float* cellinv;                        // 1 / cell size, FP32
    double* cellsz;                        // scalar: cell size of the current build
    // cached candidate pairs (built at xref with margin delta): every PT / EE
    // pair whose query box at xref overlaps the stored box inflated by
    // dhat + 2 delta; valid while every vertex stays within delta of xref
    double* xref;                          // 3 nv
    int2* cand_pt;                         // (surface vertex id, surface tri)
    int2* cand_ee;                         // (edge i, edge j), i < j
    int* cand_n;                           // device: [0] PT count, [1] EE count
    int cand_cap;                          // capacity of each list
    // pairs a grid query found and screened in FP32, finished by the list
    // kernels: one thread per pair instead of the query's thread
    int2* gpair;
    int* gpair_n;                          // device: [0] pairs appended, [1] 1 if the list overflowed
    int gpair_cap;
    // scalars
    Scalars* S;
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ double atomicMinPos(double* addr, double val) {
    // non-negative doubles order like their bit patterns
    unsigned long long* a = reinterpret_cast<unsigned long long*>(addr);
    unsigned long long v = __double_as_longlong(val);
    return __longlong_as_double(atomicMin(a, v));
}

__device__ __forceinline__ double atomicMaxPos(double* addr, double val) {
    unsigned long long* a = reinterpret_cast<unsigned long long*>(addr);
    unsigned long long v = __double_as_longlong(val);
    return __longlong_as_double(atomicMax(a, v));
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// sum over the warp, lane 0 adds to *dst
__device__ __forceinline__ void warp_add_to(double* dst, double v) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst, v);
}

__device__ __forceinline__ unsigned long long contact_key(int type, int a, int b) {
    return ((unsigned long long)type << 62) | ((unsigned long long)(unsigned)a << 31) | (unsigned long long)(unsigned)b;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

// IPC log barrier b(d) = -(d - dhat)^2 ln(d / dhat) on (0, dhat) and its
// first two derivatives (Sec. 3.1 reading).
__device__ __forceinline__ void barrier3(double d, double dhat, double& b, double& b1, double& b2) {
    if (d >= dhat) {
        b = b1 = b2 = 0.0;
        return;
    }
    if (!(d > 0.0)) {
        b = b2 = __longlong_as_double(0x7ff0000000000000ULL);
        b1 = -b;
        return;
    }
    double q = d - dhat;
    double L = log(d / dhat);
    b = -q * q * L;
    b1 = -2.0 * q * L - q * q / d;
    b2 = -2.0 * L - 4.0 * q / d + (q * q) / (d * d);
}

}  // namespace ipcb
