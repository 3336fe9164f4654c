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
#include "kernels.h"

namespace ipcb {

namespace {

constexpr int kT = 256;
inline int nblk(long long n, int t = kT) { return (int)((n + t - 1) / t); }

__host__ __device__ __forceinline__ int pk(int i, int j) { return i * 9 - (i * (i - 1)) / 2 + (j - i); }

// per vertex: g.z, g.p, g.z_prev, mass terms of the forms, |z|_inf
template <class R>
__global__ void k_forms_vert(Dev<R> D, int restart) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    double gz = 0, gp = 0, gzp = 0, zz = 0, zp = 0, pp = 0, zn = 0;
    if (v < D.nv) {
        double m = D.massd[v];
        double zsq = 0.0;
        for (int r = 0; r < 3; ++r) {
            double gi = (double)D.g[3 * v + r], zi = (double)D.z[3 * v + r], pi = restart ? 0.0 : (double)D.p[3 * v + r];
            double zpi = (double)D.zprev[3 * v + r];
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
    Scalars* S = D.S;
    warp_add_to(&S->gz, gz);
    warp_add_to(&S->gp, gp);
    warp_add_to(&S->gzprev, gzp);
    warp_add_to(&S->zHz, zz);
    warp_add_to(&S->zHp, zp);
    warp_add_to(&S->pHp, pp);
    zn = warp_max(zn);
    if ((threadIdx.x & 31) == 0 && zn > 0.0) atomicMaxPos(&S->znorm, zn);
}

template <class R>
__global__ void k_forms_tet(Dev<R> D, int restart) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    double zz = 0, zp = 0, pp = 0;
    if (t < D.nt) {
        int4 q = D.tets[t];
        int vid[4] = {q.x, q.y, q.z, q.w};
        const R* Bb = D.tetB + (size_t)(t / kPack) * 9 * kPack + (t % kPack);
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
        const R* hp = D.hess + (size_t)(t / kPack) * kH * kPack + (t % kPack);
        R Hz[9], Hp[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) Hz[i] = Hp[i] = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int j = i; j < 9; ++j) {
                R h = hp[pk(i, j) * kPack];
                Hz[i] += h * dz[j];
                Hp[i] += h * dp[j];
                if (j != i) {
                    Hz[j] += h * dz[i];
                    Hp[j] += h * dp[i];
                }
            }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            zz += (double)dz[i] * (double)Hz[i];
            zp += (double)dp[i] * (double)Hz[i];
            pp += (double)dp[i] * (double)Hp[i];
        }
    }
    Scalars* S = D.S;
    warp_add_to(&S->zHz, zz);
    warp_add_to(&S->zHp, zp);
    warp_add_to(&S->pHp, pp);
}

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

template <class R>
__global__ void k_forms_base(Dev<R> D, int restart) {
    int n = min(*D.Cb.count, D.cap);
    double zz = 0, zp = 0, pp = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double nz, np;
        rank1_dots(D.Cb.v[i], D.Cb.type[i], D.Cb.r + 3 * i, D.Cb.w + 4 * i, D.z, D.p, !restart, nz, np);
        double k = D.Cb.k[i];
        zz += k * nz * nz;
        zp += k * nz * np;
        pp += k * np * np;
    }
    Scalars* S = D.S;
    warp_add_to(&S->zHz, zz);
    warp_add_to(&S->zHp, zp);
    warp_add_to(&S->pHp, pp);
}

template <class R>
__global__ void k_forms_upd(Dev<R> D, ContactBuf C, int restart) {
    int n = min(D.S->n_upd, D.upd_cap);
    double zz = 0, zp = 0, pp = 0;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        int i = D.upd_c[u];
        double nz, np;
        rank1_dots(C.v[i], C.type[i], C.r + 3 * i, C.w + 4 * i, D.z, D.p, !restart, nz, np);
        double s = D.upd_dS[u];
        zz += s * nz * nz;
        zp += s * nz * np;
        pp += s * np * np;
    }
    Scalars* S = D.S;
    warp_add_to(&S->zHz, zz);
    warp_add_to(&S->zHp, zp);
    warp_add_to(&S->pHp, pp);
}

// (mu, nu): restart mu = g.z / z^T H~ z; else the 2x2 system of Eq. 10 with
// the singular fallback (1, 0) of supplement Eq. 20-21.
template <class R>
__global__ void k_solve2x2(Dev<R> D, int restart) {
    Scalars* S = D.S;
    double mu, nu;
    if (restart) {
        mu = S->zHz > 0.0 ? S->gz / S->zHz : 1.0;
        nu = 0.0;
    } else {
        double A11 = S->zHz, A12 = S->zHp, A22 = S->pHp;
        double b1 = S->gz, b2 = -S->gp;
        double det = A11 * A22 - A12 * A12;
        double ref = fmax(A11 * A22, D.eps_abs);
        if (!(fabs(det) >= D.eps_sing * ref)) {
            mu = 1.0;
            nu = 0.0;
        } else {
            mu = (A22 * b1 + A12 * b2) / det;
            nu = (A12 * b1 + A11 * b2) / det;
        }
    }
    if (!(mu == mu) || !(nu == nu)) S->nan_flag = 1;
    S->mu = mu;
    S->nu = nu;
}

template <class R>
__global__ void k_direction(Dev<R> D, int restart) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    double pm = 0.0, dm = 0.0;
    if (v < D.nv) {
        double mu = D.S->mu, nu = D.S->nu;
        double s = 0.0;
        for (int r = 0; r < 3; ++r) {
            double pv = restart ? 0.0 : (double)D.p[3 * v + r];
            double pn = -mu * (double)D.z[3 * v + r] + nu * pv;
            D.p[3 * v + r] = (R)pn;
            s += pn * pn;
        }
        pm = sqrt(s);
        // drift from the positions the candidate lists were built at
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
    KL(k_forms_vert<R><<<nblk(D.nv), kT, 0, st>>>(D, rs));
    KL(k_forms_tet<R><<<nblk(D.nt), kT, 0, st>>>(D, rs));
    KL(k_forms_base<R><<<296, kT, 0, st>>>(D, rs));
    KL(k_forms_upd<R><<<296, kT, 0, st>>>(D, C, rs));
}

template <class R>
void launch_direction(const Dev<R>& D, bool restart, cudaStream_t st) {
    int rs = restart ? 1 : 0;
    KL(k_solve2x2<R><<<1, 1, 0, st>>>(D, rs));
    KL(k_direction<R><<<nblk(D.nv), kT, 0, st>>>(D, rs));
}

#define INST(R)                                                                            \
    template void launch_forms<R>(const Dev<R>&, const ContactBuf&, bool, cudaStream_t); \
    template void launch_direction<R>(const Dev<R>&, bool, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace ipcb
