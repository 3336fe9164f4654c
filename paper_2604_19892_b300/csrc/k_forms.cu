// Reductions of the 2D subspace minimisation (Sec. 4.2, Eq. 9-10; supplement
// Eq. 12-22) and the direction update.
//
// The paper forms v_z = H_base z and v_p = H_base p and takes inner products.
// Here the three quadratic forms are summed element by element instead:
//   z^T H_base p = sum_v m_v z_v.p_v + sum_t (G_t z)^T K_t (G_t p)
//                + sum_{c in C_base} k_b (n_b.z)(n_b.p),
// plus (U^T z)^T (U^T p) over every classified update (supplement Eq. 12).
// One pass over the tets reads each packed Hessian once and writes nothing
// but the sums, so no scatter and no H v vector is needed.
#include <algorithm>

#include "kernels.h"

namespace ipcb {

namespace {

constexpr int kT = 256;
inline int nblk(long long n, int t = kT) { return (int)((n + t - 1) / t); }

__host__ __device__ __forceinline__ int pk(int i, int j) { return i * 9 - (i * (i - 1)) / 2 + (j - i); }


// rank-1 terms: base contacts k_b (n_b.z)(n_b.p) and updates dS (n.z)(n.p)
template <class R>
__device__ __forceinline__ void rank1_dots(const int4 q, int type, const double* r, const double* w, const R* z,
                                           const R* p, bool usep, double& nz, double& np) {
    int vid[4] = {q.x, q.y, q.z, q.w};
    int nvv = type == 2 ? 1 : 4;
    nz = 0.0;
    np = 0.0;
    for (int j = 0; j < nvv; ++j) {
        double az = r[0] * (double)z[3 * vid[j]] + r[1] * (double)z[3 * vid[j] + 1] + r[2] * (double)z[3 * vid[j] + 2];
        nz += w[j] * az;
        if (usep) {
            double ap = r[0] * (double)p[3 * vid[j]] + r[1] * (double)p[3 * vid[j] + 1] + r[2] * (double)p[3 * vid[j] + 2];
            np += w[j] * ap;
        }
    }
}

// z and p of each vertex packed into two 4-wide vectors (zp4[2v] = z,
// zp4[2v+1] = p, w = 0), so the per-tet gathers of the forms are two 16-byte
// loads per vertex; thread 0 also zeroes the iteration's reduction scalars.
template <class R>
__global__ void k_pack_zp(Dev<R> D, int restart) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v == 0) {
        Scalars* S = D.S;
        S->gz = S->gp = S->gzprev = 0.0;
        S->zHz = S->zHp = S->pHp = 0.0;
        S->znorm = 0.0;
        S->pmax = 0.0;
        S->maxdisp = 0.0;
    }
    if (v >= D.nv) return;
    V4<R>* o = reinterpret_cast<V4<R>*>(D.zp4) + 2 * v;
    o[0] = {D.z[3 * v], D.z[3 * v + 1], D.z[3 * v + 2], (R)0};
    if (restart)
        o[1] = {(R)0, (R)0, (R)0, (R)0};
    else
        o[1] = {D.p[3 * v], D.p[3 * v + 1], D.p[3 * v + 2], (R)0};
}

// (G_t z)^T K_t (G_t z), (G_t z)^T K_t (G_t p), (G_t p)^T K_t (G_t p) of one tet
// from its packed Hessian hv, rest inverse B and vertex ids, added to zz, zp, pp
template <class R>
__device__ __forceinline__ void tet_forms(const Dev<R>& D, const R hv[kH], const R B[3][3], const int vid[4], R& zz,
                                          R& zp, R& pp) {
    const V4<R>* zpk = reinterpret_cast<const V4<R>*>(D.zp4);
    V4<R> zv[4], pv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        zv[j] = zpk[2 * vid[j]];
        pv[j] = zpk[2 * vid[j] + 1];
    }
    R ez[3][3], ep[3][3];  // edge vectors x_j - x_0 of z and p
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        ez[j][0] = zv[j + 1].x - zv[0].x;
        ez[j][1] = zv[j + 1].y - zv[0].y;
        ez[j][2] = zv[j + 1].z - zv[0].z;
        ep[j][0] = pv[j + 1].x - pv[0].x;
        ep[j][1] = pv[j + 1].y - pv[0].y;
        ep[j][2] = pv[j + 1].z - pv[0].z;
    }
    R dz[9], dp[9];  // vec(dF), column-major
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            R sz = 0, sp = 0;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                sz += ez[j][r] * B[j][c];
                sp += ep[j][r] * B[j][c];
            }
            dz[3 * c + r] = sz;
            dp[3 * c + r] = sp;
        }
    R Hz[9], Hp[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) Hz[a] = Hp[a] = 0;
#pragma unroll
    for (int a = 0; a < 9; ++a)
#pragma unroll
        for (int b = a; b < 9; ++b) {
            R h = hv[pk(a, b)];
            Hz[a] += h * dz[b];
            Hp[a] += h * dp[b];
            if (b != a) {
                Hz[b] += h * dz[a];
                Hp[b] += h * dp[a];
            }
        }
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        zz += dz[a] * Hz[a];
        zp += dp[a] * Hz[a];
        pp += dp[a] * Hp[a];
    }
}

// The rest of an iteration's reductions, thread i of nth grid-stride:
// vertex terms (g.z, g.p, g.z_prev, mass terms, |z_v|), the C_base rank-1
// terms and the classified updates, added to t = {zz, zp, pp, gz, gp, gzp}
// and zn.
template <class R>
__device__ __forceinline__ void forms_rest(const Dev<R>& D, const ContactBuf& C, int restart, int i, int nth, R t[6],
                                           R& zn) {
    for (int v = i; v < D.nv; v += nth) {
        const R m = D.mass[v];
        R zsq = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            R gi = D.g[3 * v + r], zi = D.z[3 * v + r], pi = restart ? (R)0 : D.p[3 * v + r], zpi = D.zprev[3 * v + r];
            t[3] += gi * zi;
            t[4] += gi * pi;
            t[5] += gi * zpi;
            t[0] += m * zi * zi;
            t[1] += m * zi * pi;
            t[2] += m * pi * pi;
            zsq += zi * zi;
        }
        zn = fmax(zn, sqrt(zsq));
    }
    // rank-1 terms (few threads): FP64 per contact, added in R
    const int nb = min(*D.Cb.count, D.cap);
    for (int c = i; c < nb; c += nth) {
        double nz, np;
        rank1_dots(D.Cb.v[c], D.Cb.type[c], D.Cb.r + 3 * c, D.Cb.w + 4 * c, D.z, D.p, !restart, nz, np);
        double k = D.Cb.k[c];
        t[0] += (R)(k * nz * nz);
        t[1] += (R)(k * nz * np);
        t[2] += (R)(k * np * np);
    }
    const int nu = min(D.S->n_upd, D.upd_cap);
    for (int u = i; u < nu; u += nth) {
        int c = D.upd_c[u];
        double nz, np;
        rank1_dots(C.v[c], C.type[c], C.r + 3 * c, C.w + 4 * c, D.z, D.p, !restart, nz, np);
        double sd = D.upd_dS[u];
        t[0] += (R)(sd * nz * nz);
        t[1] += (R)(sd * nz * np);
        t[2] += (R)(sd * np * np);
    }
}

// Warp and block sums in R (B300's FP64 pipe is too narrow even for per-warp
// scalar work), then one FP64 atomic per block and value.
template <class R>
__device__ __forceinline__ void forms_reduce(const Dev<R>& D, R t[6], R zn) {
#pragma unroll
    for (int k = 0; k < 6; ++k) t[k] = warp_sum(t[k]);
    zn = warp_max(zn);
    __shared__ R sh[7][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) sh[k][w] = t[k];
        sh[6][w] = zn;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int k = 0; k < 6; ++k) t[k] = warp_sum(lane < nw ? sh[k][lane] : (R)0);
        R m = warp_max(lane < nw ? sh[6][lane] : (R)0);
        if (lane == 0) {
            Scalars* S = D.S;
            double* dst[6] = {&S->zHz, &S->zHp, &S->pHp, &S->gz, &S->gp, &S->gzprev};
#pragma unroll
            for (int k = 0; k < 6; ++k)
                if (t[k] != (R)0) atomicAdd(dst[k], (double)t[k]);
            if (m > (R)0) atomicMaxPos(&S->znorm, (double)m);
        }
    }
}

// One pass for all reductions of an iteration. Thread i takes tet i (all
// 45 + 9 coalesced packet loads issued before the gathers), vertex i, and,
// grid-stride, the rank-1 terms. In FP32, three CTAs per SM (85 registers a
// thread) keep the 54 packet loads of a tet in flight: 16.5 us on the
// 196,608-tet sphere pile against 18.4 us at four CTAs (64 registers). Bulk
// copies staging 4 packets per CTA, or a persistent CTA per SM streaming
// packets through a 3-stage ring, measured 20.6 us and 22.6 us: a tet moves
// 232 bytes but also gathers its vertices and does the 9x9 products, and a
// CTA's copy latency then adds to its arithmetic instead of hiding behind
// other warps' loads.
template <class R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_forms_all(Dev<R> D, ContactBuf C, int restart) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    R zz = 0, zp = 0, pp = 0;
    for (int t = i; t < D.nt; t += nth) {
        const R* hp = D.hess + (size_t)(t / kPack) * kH * kPack + (t % kPack);
        R hv[kH];
#pragma unroll
        for (int k = 0; k < kH; ++k) hv[k] = hp[k * kPack];
        const int4 q = D.tets[t];
        const int vid[4] = {q.x, q.y, q.z, q.w};
        const R* Bb = D.tetB + (size_t)(t / kPack) * 9 * kPack + (t % kPack);
        R B[3][3];
#pragma unroll
        for (int c = 0; c < 9; ++c) B[c / 3][c % 3] = Bb[c * kPack];
        tet_forms(D, hv, B, vid, zz, zp, pp);
    }
    R t[6] = {zz, zp, pp, 0, 0, 0}, zn = 0;
    forms_rest(D, C, restart, i, nth, t, zn);
    forms_reduce(D, t, zn);
}

// (mu, nu): restart mu = g.z / z^T H~ z; else the 2x2 system of Eq. 10 with
// the singular fallback (1, 0) of supplement Eq. 20-21.
__device__ __forceinline__ void solve2x2(const Scalars* S, double eps_sing, double eps_abs, int restart, double& mu,
                                         double& nu) {
    if (restart) {
        mu = S->zHz > 0.0 ? S->gz / S->zHz : 1.0;
        nu = 0.0;
    } else {
        double A11 = S->zHz, A12 = S->zHp, A22 = S->pHp;
        double b1 = S->gz, b2 = -S->gp;
        double det = A11 * A22 - A12 * A12;
        double ref = fmax(A11 * A22, eps_abs);
        if (!(fabs(det) >= eps_sing * ref)) {
            mu = 1.0;
            nu = 0.0;
        } else {
            mu = (A22 * b1 + A12 * b2) / det;
            nu = (A12 * b1 + A11 * b2) / det;
        }
    }
}

// p = -mu z + nu p with (mu, nu) from the 2x2 solve (every thread solves the
// same 2x2 from the reduced scalars; block 0 records it), max_v |p_v| and
// the drift max_v |x_v - xref_v| of the candidate lists. With FP32 bulk the
// quadratic forms carry FP32 rounding, so the singular test uses
// max(eps_sing, 1e-5) and a solution that is not a descent direction
// (g.p >= 0) takes the fallback (1, 0).
template <class R>
__global__ void k_direction(Dev<R> D, int restart) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    double mu, nu;
    const double eps_sing = sizeof(R) == 4 ? fmax(D.eps_sing, 1e-5) : D.eps_sing;
    solve2x2(D.S, eps_sing, D.eps_abs, restart, mu, nu);
    if (sizeof(R) == 4 && !restart && !(-mu * D.S->gz + nu * D.S->gp < 0.0)) {
        mu = 1.0;
        nu = 0.0;
    }
    if (v == 0) {
        if (!(mu == mu) || !(nu == nu)) D.S->nan_flag = 1;
        D.S->mu = mu;
        D.S->nu = nu;
    }
    // per vertex in the bulk precision R; |p| and the drift are rounded up
    // by a relative 1e-6 so that the FP32 bounds stay upper bounds
    const R mur = (R)(-mu), nur = (R)nu;
    R pm = 0, dm = 0;
    if (v < D.nv) {
        R s = 0;
        for (int r = 0; r < 3; ++r) {
            R pv = restart ? (R)0 : D.p[3 * v + r];
            R pn = mur * D.z[3 * v + r] + nur * pv;
            D.p[3 * v + r] = pn;
            s += pn * pn;
        }
        pm = sqrt(s);
        if (D.xref) {
            R q = 0;
            for (int r = 0; r < 3; ++r) {
                R e = (R)(D.x[3 * v + r] - D.xref[3 * v + r]);
                q += e * e;
            }
            dm = sqrt(q);
        }
    }
    pm = warp_max(pm);
    dm = warp_max(dm);
    if ((threadIdx.x & 31) == 0 && pm > (R)0) atomicMaxPos(&D.S->pmax, (1.0 + 1e-6) * (double)pm);
    if ((threadIdx.x & 31) == 0 && dm > (R)0) atomicMaxPos(&D.S->maxdisp, (1.0 + 1e-6) * (double)dm);
}

}  // namespace

template <class R>
void launch_forms_prep(const Dev<R>& D, bool restart, cudaStream_t st) {
    KL(k_pack_zp<R><<<nblk(std::max(D.nv, 1)), kT, 0, st>>>(D, restart ? 1 : 0));
}

template <class R>
void launch_forms_main(const Dev<R>& D, const ContactBuf& C, bool restart, cudaStream_t st) {
    KL(k_forms_all<R><<<nblk(std::max(std::max(D.nt, D.nv), 1)), kT, 0, st>>>(D, C, restart ? 1 : 0));
}

template <class R>
void launch_forms(const Dev<R>& D, const ContactBuf& C, bool restart, cudaStream_t st) {
    launch_forms_prep(D, restart, st);
    launch_forms_main(D, C, restart, st);
}

template <class R>
void launch_direction(const Dev<R>& D, bool restart, cudaStream_t st) {
    int rs = restart ? 1 : 0;
    KL(k_direction<R><<<nblk(std::max(D.nv, 1)), kT, 0, st>>>(D, rs));
}

#define INST(R)                                                                            \
    template void launch_forms<R>(const Dev<R>&, const ContactBuf&, bool, cudaStream_t); \
    template void launch_forms_prep<R>(const Dev<R>&, bool, cudaStream_t);                \
    template void launch_forms_main<R>(const Dev<R>&, const ContactBuf&, bool, cudaStream_t); \
    template void launch_direction<R>(const Dev<R>&, bool, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace ipcb
