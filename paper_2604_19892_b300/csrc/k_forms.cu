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

// One pass for all reductions of an iteration. Thread i takes tet i (the
// stored projected Hessian: (G_t z)^T K_t (G_t p) and the like), vertex i
// (g.z, g.p, g.z_prev, mass terms, |z_v|), and, grid-stride, the C_base
// rank-1 terms and the classified updates. Per-thread values are in the
// bulk precision R (contact terms in FP64); each warp sums in R, the warps'
// partials are summed in FP64 with one atomic per block and value.
template <class R>
__global__ void __launch_bounds__(256) k_forms_all(Dev<R> D, ContactBuf C, int restart) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;
    R zz = 0, zp = 0, pp = 0, gz = 0, gp = 0, gzp = 0, zn = 0;
    if (i < D.nt) {
        int4 q = D.tets[i];
        int vid[4] = {q.x, q.y, q.z, q.w};
        const R* Bb = D.tetB + (size_t)(i / kPack) * 9 * kPack + (i % kPack);
        R B[3][3];
#pragma unroll
        for (int c = 0; c < 9; ++c) B[c / 3][c % 3] = Bb[c * kPack];
        R dz[9], dp[9];  // vec(dF), column-major
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                R sz = 0, sp = 0;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    sz += (D.z[3 * vid[j + 1] + r] - D.z[3 * vid[0] + r]) * B[j][c];
                    if (!restart) sp += (D.p[3 * vid[j + 1] + r] - D.p[3 * vid[0] + r]) * B[j][c];
                }
                dz[3 * c + r] = sz;
                dp[3 * c + r] = sp;
            }
        const R* hp = D.hess + (size_t)(i / kPack) * kH * kPack + (i % kPack);
        R Hz[9], Hp[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) Hz[a] = Hp[a] = 0;
#pragma unroll
        for (int a = 0; a < 9; ++a)
#pragma unroll
            for (int b = a; b < 9; ++b) {
                R h = hp[pk(a, b) * kPack];
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
    if (i < D.nv) {
        const R m = D.mass[i];
        R zsq = 0;
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            R gi = D.g[3 * i + r], zi = D.z[3 * i + r], pi = restart ? (R)0 : D.p[3 * i + r], zpi = D.zprev[3 * i + r];
            gz += gi * zi;
            gp += gi * pi;
            gzp += gi * zpi;
            zz += m * zi * zi;
            zp += m * zi * pi;
            pp += m * pi * pi;
            zsq += zi * zi;
        }
        zn = sqrt(zsq);
    }
    double czz = 0, czp = 0, cpp = 0;
    const int nb = min(*D.Cb.count, D.cap);
    for (int c = i; c < nb; c += nth) {
        double nz, np;
        rank1_dots(D.Cb.v[c], D.Cb.type[c], D.Cb.r + 3 * c, D.Cb.w + 4 * c, D.z, D.p, !restart, nz, np);
        double k = D.Cb.k[c];
        czz += k * nz * nz;
        czp += k * nz * np;
        cpp += k * np * np;
    }
    const int nu = min(D.S->n_upd, D.upd_cap);
    for (int u = i; u < nu; u += nth) {
        int c = D.upd_c[u];
        double nz, np;
        rank1_dots(C.v[c], C.type[c], C.r + 3 * c, C.w + 4 * c, D.z, D.p, !restart, nz, np);
        double sd = D.upd_dS[u];
        czz += sd * nz * nz;
        czp += sd * nz * np;
        cpp += sd * np * np;
    }
    // warp sums: bulk terms in R, contact terms in FP64 (zero in most warps)
    zz = warp_sum(zz);
    zp = warp_sum(zp);
    pp = warp_sum(pp);
    gz = warp_sum(gz);
    gp = warp_sum(gp);
    gzp = warp_sum(gzp);
    zn = warp_max(zn);
    const bool any_c = __any_sync(0xffffffffu, czz != 0.0 || czp != 0.0 || cpp != 0.0);
    if (any_c) {
        czz = warp_sum(czz);
        czp = warp_sum(czp);
        cpp = warp_sum(cpp);
    }
    __shared__ double sh[6][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][w] = (double)zz + czz;
        sh[1][w] = (double)zp + czp;
        sh[2][w] = (double)pp + cpp;
        sh[3][w] = (double)gz;
        sh[4][w] = (double)gp;
        sh[5][w] = (double)gzp;
        if (zn > (R)0) atomicMaxPos(&D.S->znorm, (double)zn);
    }
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        double t[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) t[k] = warp_sum(lane < nw ? sh[k][lane] : 0.0);
        if (lane == 0) {
            Scalars* S = D.S;
            double* dst[6] = {&S->zHz, &S->zHp, &S->pHp, &S->gz, &S->gp, &S->gzprev};
#pragma unroll
            for (int k = 0; k < 6; ++k)
                if (t[k] != 0.0) atomicAdd(dst[k], t[k]);
        }
    }
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
    double pm = 0.0, dm = 0.0;
    if (v < D.nv) {
        double s = 0.0;
        for (int r = 0; r < 3; ++r) {
            double pv = restart ? 0.0 : (double)D.p[3 * v + r];
            double pn = -mu * (double)D.z[3 * v + r] + nu * pv;
            D.p[3 * v + r] = (R)pn;
            s += pn * pn;
        }
        pm = sqrt(s);
        if (D.xref) {
            double q = 0.0;
            for (int r = 0; r < 3; ++r) {
                double e = D.x[3 * v + r] - D.xref[3 * v + r];
                q += e * e;
            }
            dm = sqrt(q);
        }
    }
    pm = warp_max(pm);
    dm = warp_max(dm);
    if ((threadIdx.x & 31) == 0 && pm > 0.0) atomicMaxPos(&D.S->pmax, pm);
    if ((threadIdx.x & 31) == 0 && dm > 0.0) atomicMaxPos(&D.S->maxdisp, dm);
}

}  // namespace

template <class R>
void launch_forms(const Dev<R>& D, const ContactBuf& C, bool restart, cudaStream_t st) {
    int rs = restart ? 1 : 0;
    launch_zero_scalars(D, st);
    KL(k_forms_all<R><<<nblk(std::max(std::max(D.nt, D.nv), 1)), kT, 0, st>>>(D, C, rs));
}

template <class R>
void launch_direction(const Dev<R>& D, bool restart, cudaStream_t st) {
    int rs = restart ? 1 : 0;
    KL(k_direction<R><<<nblk(std::max(D.nv, 1)), kT, 0, st>>>(D, rs));
}

#define INST(R)                                                                            \
    template void launch_forms<R>(const Dev<R>&, const ContactBuf&, bool, cudaStream_t); \
    template void launch_direction<R>(const Dev<R>&, bool, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace ipcb
