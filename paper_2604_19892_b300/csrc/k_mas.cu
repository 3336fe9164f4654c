// MAS preconditioner (Sec. 3.3; supplement Eq. 1-4), its restart rebuild, and
// the Sparse-Input Woodbury update of the level-0 inverses (Sec. 4.1, Eq. 7-8).
//
// RebuildMAS at x:
//  1. per tet: dP/dF (9x9) of the SNH density, PSD-projected through its
//     closed-form eigensystem (negative eigenvalues clamped), times h^2 V,
//     stored packed (45 values);
//  2. level blocks of H_base = M + h^2 sum_t K_t + sum_{c in C} k n n^T:
//     level 0 takes the 3x3 couplings between vertices of one subdomain;
//     level l >= 1 takes C_l H C_l^T restricted to one level-l subdomain.
//     Elastic and PT/EE contact terms annihilate rigid translations, so a
//     term whose vertices all fall in one level-l node adds nothing to that
//     level and is skipped; mass and point-ground terms always add;
//  3. every 96x96 block is inverted through a scaled Cholesky factorisation
//     in register tiles (B = s W^T W s, W = L^{-1}) and kept as the packed
//     lower triangular factor W' = W diag(s), B = W'^T W'; padded slots carry
//     an identity;
//  4. the contact set is snapshot as C_base with a key table.
// Woodbury (non-restart iterations): each current contact is classified
// against C_base (new / rotated: dS = k, u = sqrt(k) n; stiffer: dS = k - k_b,
// u = sqrt(dS) n; softer: skipped); every subdomain keeps the K updates of
// largest dS (ties by ascending key) touching it; the block apply reads W'_d
// once, forms V = W' [g_d, U_d], the K x K capacitance C = I + V_U^T V_U (=
// I + U^T B U) and r = V_U^T V_g (= U^T B g), solves C lambda = r in FP64 and
// returns z_d = W'^T (V_g - V_U lambda) = B g_d - B U lambda (Eq. 7).  Coarse
// levels stay frozen (Eq. 8).
#include <algorithm>
#include <vector>
#include <type_traits>

#include <cuda_bf16.h>

#include "bulk.cuh"
#include "kernels.h"

namespace ipcb {

namespace {

constexpr int kT = 128;
constexpr int kCon = 12;  // values per coarse assembly record: a 3x3 block, padded to 16 bytes
inline int nblk(long long n, int t = kT) { return (int)((n + t - 1) / t); }

__host__ __device__ __forceinline__ int pk(int i, int j) {  // packed upper index, i <= j
    return i * 9 - (i * (i - 1)) / 2 + (j - i);
}

// FP64 -> FP32, rounded to nearest (ties to even), on the integer pipes: the
// IEEE 754 binary64 fields are re-packed as binary32 (exponent bias 1023 ->
// 127, the 52-bit fraction rounded to 23 bits; a carry out of the fraction
// raises the exponent, as the format intends). Handles zeros and magnitudes
// within 2^+-100 and returns true; otherwise returns false and leaves f
// unset. B300's FP64 pipe (conversions included) runs at a small fraction
// of its integer rate.
__device__ __forceinline__ bool f64_to_f32_rn(double x, float& f) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned ex = (unsigned)(bits >> 52) & 0x7FFu;
    if ((bits << 1) == 0ULL) {
        f = 0.f;
        return true;
    }
    if (ex < 1023u - 100u || ex > 1023u + 100u) return false;
    const unsigned long long frac = bits & ((1ULL << 52) - 1ULL);
    unsigned m = (unsigned)(frac >> 29);
    const unsigned rest = (unsigned)frac & ((1u << 29) - 1u);
    const unsigned half = 1u << 28;
    m += (rest > half || (rest == half && (m & 1u))) ? 1u : 0u;
    f = __uint_as_float(((unsigned)(bits >> 32) & 0x80000000u) + ((ex - 1023u + 127u) << 23) + m);
    return true;
}
__device__ __forceinline__ float to_f32(double x) {
    float f;
    return f64_to_f32_rn(x, f) ? f : (float)x;
}

template <class R>
__device__ __forceinline__ void load_B(const Dev<R>& D, int t, R B[3][3]) {
    const R* base = D.tetB + (size_t)(t / kPack) * 9 * kPack + (t % kPack);
#pragma unroll
    for (int c = 0; c < 9; ++c) B[c / 3][c % 3] = base[c * kPack];
}

// ------------------------------------------------------ per-tet projected Hessian

// Cyclic Jacobi on a symmetric 3x3 matrix: eigenvalues on the diagonal of
// A, eigenvectors in the columns of V.
template <class R>
__device__ __forceinline__ void sym3_jacobi(R A[3][3], R V[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? (R)1 : (R)0;
    R fro = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) fro += A[i][j] * A[i][j];
    const R tol = (sizeof(R) == 8 ? (R)1e-32 : (R)1e-14) * fro;
#pragma unroll 1
    for (int sweep = 0; sweep < 12; ++sweep) {
        if (A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2] <= tol) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int pp = pq == 2 ? 1 : 0, qq = pq == 0 ? 1 : 2;
            R apq = A[pp][qq];
            if (apq == (R)0) continue;
            R th = (A[qq][qq] - A[pp][pp]) / (2 * apq);
            R tt = (th >= 0 ? (R)1 : (R)-1) / (fabs(th) + sqrt(th * th + (R)1));
            R c = (R)1 / sqrt(tt * tt + (R)1), sn = tt * c;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                R akp = A[k][pp], akq = A[k][qq];
                A[k][pp] = c * akp - sn * akq;
                A[k][qq] = sn * akp + c * akq;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                R apk = A[pp][k], aqk = A[qq][k];
                A[pp][k] = c * apk - sn * aqk;
                A[qq][k] = sn * apk + c * aqk;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                R vkp = V[k][pp], vkq = V[k][qq];
                V[k][pp] = c * vkp - sn * vkq;
                V[k][qq] = sn * vkp + c * vkq;
            }
        }
    }
}

template <class R>
__device__ __forceinline__ void add_mode(R acc[kH], R e, const R q[9]) {
    if (!(e > (R)0)) return;
    int k = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        R ei = e * q[i];
#pragma unroll
        for (int j = i; j < 9; ++j) acc[k++] += ei * q[j];
    }
}

// Per tet: K_t = h^2 V (d^2 Psi / dF^2)^+ in F space (vec column-major),
// Psi = mu/2 (|F|^2 - 3) - mu (J - 1) + lam/2 (J - 1)^2, so
// d^2 Psi/dF^2 = mu I + lam g g^T + (lam (J - 1) - mu) d^2 J/dF^2, g = cof F.
// Its eigensystem is taken in closed form from the rotation-signed SVD
// F = U diag(s) V^T (the analytic eigensystems of isotropic energies,
// Smith et al. 2019): in the frame, d^2 J/dF^2 has eigenvalue +s_k on the
// twist (E_ab - E_ba)/sqrt2 and -s_k on the flip (E_ab + E_ba)/sqrt2 of the
// index pair {a, b} without k, and acts on the scaling modes diag(w) as
// [[0, s2, s1], [s2, 0, s0], [s1, s0, 0]]; g lies in the scaling modes as
// (s1 s2, s0 s2, s0 s1). The projection keeps the positive eigenvalues; it
// equals the clamped 9x9 eigen-decomposition up to rounding (the projection
// onto the PSD cone does not depend on the basis chosen within a cluster).
template <class R>
__global__ void __launch_bounds__(64) k_tet_hessian(Dev<R> D, const double* __restrict__ x) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= D.nt) return;
    int4 q4 = D.tets[t];
    int vid[4] = {q4.x, q4.y, q4.z, q4.w};
    R B[3][3];
    load_B(D, t, B);
    R F[3][3];
    if constexpr (sizeof(R) == 4) {
        // edge vectors exact in FP64, rounded to FP32; F in FP32 like the rest
        // of this Hessian
        float Ds[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j) Ds[r][j] = to_f32(x[3 * vid[j + 1] + r] - x[3 * vid[0] + r]);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) F[r][c] = Ds[r][0] * B[0][c] + Ds[r][1] * B[1][c] + Ds[r][2] * B[2][c];
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double sacc = 0.0;
                for (int j = 0; j < 3; ++j) sacc += (x[3 * vid[j + 1] + r] - x[3 * vid[0] + r]) * (double)B[j][c];
                F[r][c] = (R)sacc;
            }
    }
    const R J = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
    // V, s^2 from F^T F, sorted descending, V a rotation
    R C[3][3], V[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) C[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
    sym3_jacobi(C, V);
    R w[3] = {C[0][0], C[1][1], C[2][2]};
    auto swapc = [&](int a, int b) {
        R tw = w[a];
        w[a] = w[b];
        w[b] = tw;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            R tv = V[k][a];
            V[k][a] = V[k][b];
            V[k][b] = tv;
        }
    };
    if (w[0] < w[1]) swapc(0, 1);
    if (w[1] < w[2]) swapc(1, 2);
    if (w[0] < w[1]) swapc(0, 1);
    R detV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) - V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
             V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
    if (detV < (R)0)
#pragma unroll
        for (int k = 0; k < 3; ++k) V[k][2] = -V[k][2];
    // U by Gram-Schmidt on the columns of F V; u2 = u0 x u1 keeps U a rotation
    R b[3][3];  // b[i] = F v_i
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int r = 0; r < 3; ++r) b[i][r] = F[r][0] * V[0][i] + F[r][1] * V[1][i] + F[r][2] * V[2][i];
    R U[3][3], sg[3];
    R n0 = sqrt(b[0][0] * b[0][0] + b[0][1] * b[0][1] + b[0][2] * b[0][2]);
    R u0[3], u1[3], u2[3];
    if (n0 > (R)0) {
        for (int r = 0; r < 3; ++r) u0[r] = b[0][r] / n0;
    } else {
        u0[0] = 1;
        u0[1] = u0[2] = 0;
    }
    R d01 = u0[0] * b[1][0] + u0[1] * b[1][1] + u0[2] * b[1][2];
    for (int r = 0; r < 3; ++r) u1[r] = b[1][r] - d01 * u0[r];
    R n1 = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
    if (n1 > (R)(sizeof(R) == 8 ? 1e-150 : 1e-30)) {
        for (int r = 0; r < 3; ++r) u1[r] /= n1;
    } else {
        // any unit vector orthogonal to u0
        int ax = fabs(u0[0]) <= fabs(u0[1]) ? (fabs(u0[0]) <= fabs(u0[2]) ? 0 : 2) : (fabs(u0[1]) <= fabs(u0[2]) ? 1 : 2);
        R e[3] = {0, 0, 0};
        e[ax] = 1;
        u1[0] = u0[1] * e[2] - u0[2] * e[1];
        u1[1] = u0[2] * e[0] - u0[0] * e[2];
        u1[2] = u0[0] * e[1] - u0[1] * e[0];
        R m = sqrt(u1[0] * u1[0] + u1[1] * u1[1] + u1[2] * u1[2]);
        for (int r = 0; r < 3; ++r) u1[r] /= m;
        n1 = 0;
    }
    u2[0] = u0[1] * u1[2] - u0[2] * u1[1];
    u2[1] = u0[2] * u1[0] - u0[0] * u1[2];
    u2[2] = u0[0] * u1[1] - u0[1] * u1[0];
    sg[0] = n0;
    sg[1] = n1;
    sg[2] = u2[0] * b[2][0] + u2[1] * b[2][1] + u2[2] * b[2][2];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        U[r][0] = u0[r];
        U[r][1] = u1[r];
        U[r][2] = u2[r];
    }
    const R mu = sizeof(R) == 4 ? (R)to_f32(D.tet_mu[t]) : (R)D.tet_mu[t];
    const R lam = sizeof(R) == 4 ? (R)to_f32(D.tet_lam[t]) : (R)D.tet_lam[t];
    const R cJ = lam * (J - (R)1) - mu;
    R acc[kH];
#pragma unroll
    for (int k = 0; k < kH; ++k) acc[k] = 0;
    const R r2 = (R)0.70710678118654752440;
    R q[9];
    // twist / flip modes of the index pairs {1,2}, {0,2}, {0,1}
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int a = k == 0 ? 1 : 0, bb = k == 2 ? 1 : 2;
#pragma unroll
        for (int flip = 0; flip < 2; ++flip) {
            const R sgn = flip ? (R)1 : (R)-1;
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int r = 0; r < 3; ++r) q[3 * c + r] = r2 * (U[r][a] * V[c][bb] + sgn * U[r][bb] * V[c][a]);
            add_mode(acc, flip ? mu - cJ * sg[k] : mu + cJ * sg[k], q);
        }
    }
    // scaling modes: mu I + lam gh gh^T + cJ S on diag(w)
    R As[3][3], Ws[3][3];
    const R gh[3] = {sg[1] * sg[2], sg[0] * sg[2], sg[0] * sg[1]};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) As[i][j] = lam * gh[i] * gh[j] + (i == j ? mu : (R)0);
    As[0][1] += cJ * sg[2];
    As[1][0] += cJ * sg[2];
    As[0][2] += cJ * sg[1];
    As[2][0] += cJ * sg[1];
    As[1][2] += cJ * sg[0];
    As[2][1] += cJ * sg[0];
    sym3_jacobi(As, Ws);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int r = 0; r < 3; ++r)
                q[3 * c + r] = U[r][0] * Ws[0][m] * V[c][0] + U[r][1] * Ws[1][m] * V[c][1] + U[r][2] * Ws[2][m] * V[c][2];
        add_mode(acc, As[m][m], q);
    }
    const R scl = (R)(D.h * D.h * D.tet_vol[t]);
    R* out = D.hess + (size_t)(t / kPack) * kH * kPack + (t % kPack);
#pragma unroll
    for (int k = 0; k < kH; ++k) out[k * kPack] = scl * acc[k];
}

// ------------------------------------------------------ block assembly

// Every assembly block set to its mass term: zero except the lumped node
// masses on the diagonal (a table fixed by the mesh), level 0 into asmb (at
// and below the diagonal), the coarse levels into asmbc. Four FP64 entries
// (two 16-byte stores) per thread and step; only diagonal rows read the
// table.
template <class R>
__global__ void __launch_bounds__(256) k_init_blocks(Dev<R> D, int nb0, int nb) {
    constexpr int kQ = kBlk * kBlk / 4;  // 4-entry groups per block
    const int n4 = nb * kQ;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n4; e += gridDim.x * blockDim.x) {
        const int b = e / kQ;
        const int rem = 4 * (e - b * kQ);
        const int row = rem / kBlk, col = rem - row * kBlk;
        const int dc = row - col;  // the diagonal sits at entry dc of this group if 0 <= dc < 4
        // level 0 is assembled and read at or below the diagonal only: its
        // groups strictly above it were zeroed once at scene set-up and stay 0
        if (b < nb0 && dc < 0) continue;
        const double dg = (dc >= 0 && dc < 4) ? D.mdiag[(size_t)b * kBlk + row] : 0.0;
        double* dst = (b < nb0 ? D.asmb + (size_t)b * (kBlk * kBlk) : D.asmbc + (size_t)(b - nb0) * (kBlk * kBlk)) + rem;
        reinterpret_cast<double2*>(dst)[0] = make_double2(dc == 0 ? dg : 0.0, dc == 1 ? dg : 0.0);
        reinterpret_cast<double2*>(dst)[1] = make_double2(dc == 2 ? dg : 0.0, dc == 3 ? dg : 0.0);
    }
}

// Elastic terms h^2 K_t of every tet, K_t = G^T H G with G the 9x12 map from
// the four vertex displacements to dF (rows Bf[a], Bf[0] = -sum of the rest).
// Level 0 takes the 3x3 blocks K_ab = sum_{c,c2} Bf[a][c] H[3c+r][3c2+s] Bf[b][c2]
// of the vertex pairs inside one subdomain, with FP64 atomics (a vertex pair
// is shared by a few tets only: 24 at most on the sphere pile).
template <class R>
__global__ void k_assemble_tets0(Dev<R> D) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= D.nt) return;
    const int4 q = D.tets[t];
    const int vid[4] = {q.x, q.y, q.z, q.w};
    int g[4], sl[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        g[a] = D.grp0[vid[a]];
        sl[a] = D.slot0[vid[a]];
    }
    R Bm[3][3];
    load_B(D, t, Bm);
    R Bf[4][3];
    for (int c = 0; c < 3; ++c) {
        Bf[0][c] = -(Bm[0][c] + Bm[1][c] + Bm[2][c]);
        for (int j = 0; j < 3; ++j) Bf[j + 1][c] = Bm[j][c];
    }
    const R* hp = D.hess + (size_t)(t / kPack) * kH * kPack + (t % kPack);
    R H[9][9];
    for (int i = 0; i < 9; ++i)
        for (int j = i; j < 9; ++j) {
            R v = hp[pk(i, j) * kPack];
            H[i][j] = v;
            H[j][i] = v;
        }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        R HB[9][3];
        for (int i = 0; i < 9; ++i)
            for (int s2 = 0; s2 < 3; ++s2) {
                R inner = 0;
                for (int c2 = 0; c2 < 3; ++c2) inner += H[i][3 * c2 + s2] * Bf[b][c2];
                HB[i][s2] = inner;
            }
        // lower triangle only: both inversion kernels read a block's entries
        // at or below the diagonal and nothing else reads level-0 blocks, so
        // a pair of distinct vertices adds its 3x3 block once (row slot >
        // column slot) and a vertex its own block's lower half: 78 FP64
        // atomics per tet instead of 144
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            if (g[a] != g[b] || sl[a] < sl[b]) continue;
            const bool self = a == b;
            double* A = D.asmb + (size_t)g[a] * (kBlk * kBlk) + (3 * sl[a]) * kBlk + 3 * sl[b];
            for (int r = 0; r < 3; ++r)
                for (int s2 = 0; s2 < 3; ++s2) {
                    if (self && s2 > r) continue;
                    R acc = 0;
                    for (int c = 0; c < 3; ++c) acc += Bf[a][c] * HB[3 * c + r][s2];
                    atomicAdd(&A[r * kBlk + s2], (double)acc);
                }
        }
    }
}

// Coarse levels. At level l the Galerkin block of nodes P, Q sums the level-0
// blocks of their vertices, (sum_{a in P} Bf[a])^T H (sum_{b in Q} Bf[b]) in
// the same 3x3 sense, and a tet inside one node adds nothing (its rows sum to
// zero). The mesh fixes which (tet, vertex set P, vertex set Q) reach which
// target 3x3 block (coarse block, node slot i <= node slot j), so the host
// lists these contributions once, sorted by target. The assembly is then two
// passes: one thread per tet writes each of its contributions to its slot of
// a value array (one 16-byte aligned record of kCon values each), and one
// warp per target (long targets cut into chunks, added atomically) sums its
// contiguous run and adds the block and its transpose.
template <class R>
__global__ void k_asm_contrib(Dev<R> D) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= D.nt) return;
    const int e0 = D.tcon_off[t], e1 = D.tcon_off[t + 1];
    R Bm[3][3];
    load_B(D, t, Bm);
    R b0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) b0[c] = -(Bm[0][c] + Bm[1][c] + Bm[2][c]);
    const R* hp = D.hess + (size_t)(t / kPack) * kH * kPack + (t % kPack);
    R H[9][9];
#pragma unroll
    for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = i; j < 9; ++j) {
            const R v = hp[pk(i, j) * kPack];
            H[i][j] = v;
            H[j][i] = v;
        }
    int2 nxt = e0 < e1 ? D.tcon[e0] : make_int2(0, 0);
    for (int e = e0; e < e1; ++e) {
        const int2 c = nxt;
        if (e + 1 < e1) nxt = D.tcon[e + 1];
        const int mk = c.y;
        R BA[3], BB[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            BA[k] = ((mk & 1) ? b0[k] : (R)0) + ((mk & 2) ? Bm[0][k] : (R)0) + ((mk & 4) ? Bm[1][k] : (R)0) +
                    ((mk & 8) ? Bm[2][k] : (R)0);
            BB[k] = ((mk & 16) ? b0[k] : (R)0) + ((mk & 32) ? Bm[0][k] : (R)0) + ((mk & 64) ? Bm[1][k] : (R)0) +
                    ((mk & 128) ? Bm[2][k] : (R)0);
        }
        R HB[9][3];
#pragma unroll
        for (int i = 0; i < 9; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) HB[i][k] = H[i][k] * BB[0] + H[i][3 + k] * BB[1] + H[i][6 + k] * BB[2];
        R K[12];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) K[3 * r + k] = BA[0] * HB[r][k] + BA[1] * HB[3 + r][k] + BA[2] * HB[6 + r][k];
        K[9] = K[10] = K[11] = (R)0;
        V4<R>* out = reinterpret_cast<V4<R>*>(D.cval + (size_t)kCon * c.x);
#pragma unroll
        for (int q = 0; q < 3; ++q) out[q] = V4<R>{K[4 * q], K[4 * q + 1], K[4 * q + 2], K[4 * q + 3]};
    }
}

template <class R>
__global__ void __launch_bounds__(256) k_asm_sum(Dev<R> D) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;  // one warp per item
    const int lane = threadIdx.x & 31;
    if (i >= D.nitem) return;
    const int4 it = D.item[i];  // coarse block, slot i, slot j | split << 8, first entry
    const int end = D.item[i + 1].w;
    R acc[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = 0;
    for (int e = it.w + lane; e < end; e += 32) {
        const V4<R>* in = reinterpret_cast<const V4<R>*>(D.cval + (size_t)kCon * e);
        const V4<R> a = in[0], b = in[1], c = in[2];
        acc[0] += a.x;
        acc[1] += a.y;
        acc[2] += a.z;
        acc[3] += a.w;
        acc[4] += b.x;
        acc[5] += b.y;
        acc[6] += b.z;
        acc[7] += b.w;
        acc[8] += c.x;
    }
#pragma unroll
    for (int q = 0; q < 9; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    const int si = it.y, sj = it.z & 0xff;
    const bool split = (it.z >> 8) != 0;
    double* A = D.asmbc + (size_t)it.x * (kBlk * kBlk);
    // lanes 0-8 take one entry each (and its transpose)
    if (lane < 9) {
        const int r = lane / 3, k = lane - 3 * r;
        R v = acc[0];
#pragma unroll
        for (int q = 1; q < 9; ++q)
            if (q == lane) v = acc[q];
        double* p0 = A + (3 * si + r) * kBlk + 3 * sj + k;
        double* p1 = A + (3 * sj + k) * kBlk + 3 * si + r;
        if (split) {
            atomicAdd(p0, (double)v);
            if (si != sj) atomicAdd(p1, (double)v);
        } else {
            // the only writer of these entries in this kernel
            *p0 += (double)v;
            if (si != sj) *p1 += (double)v;
        }
    }
}

// Contact terms kappa b''(d) grad d grad d^T (Eq. 1, Alg. 1), in FP64 with
// FP64 atomics (their stiffness spans many orders of magnitude, and their
// weights cancel at the coarse levels). Level 0 takes the vertex pairs inside
// one subdomain; a coarse level sums the weights of the vertices sharing a
// node, W_P = sum_{a in P} w_a, and adds k W_P W_Q r r^T per node pair (none
// for a pair or edge contact inside one node: its weights sum to zero).
__device__ __forceinline__ void add_rr(double* A, int si, int sj, const double kr[3][3], double c,
                                       bool lower = false) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s2 = 0; s2 < 3; ++s2) {
            if (lower && si == sj && s2 > r) continue;  // above the diagonal of a diagonal 3x3 block
            const double v = c * kr[r][s2];
            if (v != 0.0) atomicAdd(&A[(3 * si + r) * kBlk + 3 * sj + s2], v);
        }
}

template <class R>
__global__ void k_assemble_contacts(Dev<R> D, ContactBuf C) {
    const int n = min(*C.count, D.cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int4 q = C.v[i];
        const int vid[4] = {q.x, q.y, q.z, q.w};
        const int nvv = C.type[i] == 2 ? 1 : 4;
        const double k = C.k[i];
        const double r[3] = {C.r[3 * i], C.r[3 * i + 1], C.r[3 * i + 2]};
        const double w[4] = {C.w[4 * i], C.w[4 * i + 1], C.w[4 * i + 2], C.w[4 * i + 3]};
        double kr[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) kr[a][b] = k * r[a] * r[b];
        int g[4], sl[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            g[a] = a < nvv ? D.grp0[vid[a]] : -1;
            sl[a] = a < nvv ? D.slot0[vid[a]] : 0;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b)
                // level 0 at and below the diagonal only (row slot >= column
                // slot): the blocks of (a, b) and (b, a) are transposes
                if (a < nvv && b < nvv && g[a] == g[b] && sl[a] >= sl[b])
                    add_rr(D.asmb + (size_t)g[a] * (kBlk * kBlk), sl[a], sl[b], kr, w[a] * w[b], true);
        for (int l = 1; l < D.nlev; ++l) {
            if (nvv == 1) {
                // a point-ground contact adds k n n^T (weight 1, the plane
                // normal n) to its node's diagonal block: its stiffness is
                // summed per node here and the block updated once per node
                // (k_assemble_pg_coarse), instead of nine atomics per contact
                // on the few entries that every ground contact of a coarse
                // node shares
                atomicAdd(&D.pg_k[D.coarse_off[l] / 3 + D.node_of_vert[l][vid[0]]], k);
                continue;
            }
            int nd[4];
            double W[4] = {0.0, 0.0, 0.0, 0.0};
            int m = 0;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                if (a >= nvv) break;
                const int nn = D.node_of_vert[l][vid[a]];
                int kk = m;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u < m && nd[u] == nn && kk == m) kk = u;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (u == kk) {
                        if (kk == m) nd[u] = nn;
                        W[u] += w[a];
                    }
                if (kk == m) ++m;
            }
            if (nvv == 4 && m == 1) continue;
            double* Ab = D.asmbc + (size_t)(D.blk_off[l] - D.blk_off[1]) * (kBlk * kBlk);
            int ng[4], ns[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                ng[u] = u < m ? D.grp_of_node[l][nd[u]] : -1;
                ns[u] = u < m ? D.slot_of_node[l][nd[u]] : 0;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    if (u < m && v < m && ng[u] == ng[v])
                        add_rr(Ab + (size_t)ng[u] * (kBlk * kBlk), ns[u], ns[v], kr, W[u] * W[v]);
        }
    }
}

// the summed point-ground stiffness K of each coarse node: K n n^T on its
// diagonal 3x3 block (one thread per node, the only writer of those entries
// in this kernel; the contact assembly before it has finished)
template <class R>
__global__ void k_assemble_pg_coarse(Dev<R> D) {
    const int n = D.coarse_off[D.nlev] / 3;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double k = D.pg_k[i];
        if (k == 0.0) continue;
        int l = 1;
        while (l + 1 < D.nlev && i >= D.coarse_off[l + 1] / 3) ++l;
        const int node = i - D.coarse_off[l] / 3;
        const int s = D.slot_of_node[l][node];
        double* A = D.asmbc + (size_t)(D.blk_off[l] - D.blk_off[1] + D.grp_of_node[l][node]) * (kBlk * kBlk);
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) A[(3 * s + r) * kBlk + 3 * s + c] += k * D.gn[r] * D.gn[c];
    }
}

// ------------------------------------------------------ batched inversion

// Inverse of one SPD 96x96 subdomain block, B_d = M_d^{-1} (Sec. 4.2), one
// CTA per block. The block is scaled to a unit diagonal, S = s A s with
// s = diag(A)^{-1/2}; S = L L^T by right-looking Cholesky; W = L^{-1}; and
// B = s W^T W s, kept as its factor W' = W diag(s). Each pivot is floored at
// eps_piv of the unit diagonal (the pivot relative to the original diagonal
// entry) and raised where needed to keep every L_rk^2 <= 1: a numerically
// singular block (stiff rank-1 contact terms) is replaced by A plus a small
// non-negative diagonal shift. B = W'^T W' is symmetric positive
// semi-definite whatever the rounding of W', so it remains a valid
// preconditioner when R is FP32.
//
// Register tiling: the lower triangle is cut into 6x6 tiles (136 of them),
// one per thread. Each elimination step broadcasts one column of L (or one
// row of W) through shared memory; the broadcast vector is double-buffered
// by step parity so a step needs a single barrier.
constexpr int kTile = 6;
constexpr int kNT = kBlk / kTile;                // 16 tiles per side
constexpr int kNTiles = kNT * (kNT + 1) / 2;     // 136
constexpr int kInvThreads = 160;
static_assert(kNT * kTile == kBlk, "tile size must divide the block size");
static_assert(kInvThreads >= kNTiles && kInvThreads % 32 == 0, "one thread per lower tile");

// Packed lower column panels: panel kt holds columns 6 kt .. 6 kt + 5 of a
// lower-triangular 96 x 96 matrix over rows 6 kt .. 95, column-major (each
// column is 96 - 6 kt consecutive entries): 4,896 entries, about half the
// square. A 6-row slice of a column starts at an even index.
__host__ __device__ constexpr int panel_off(int kt) { return kTile * (kBlk * kt - kTile * kt * (kt - 1) / 2); }
constexpr int kPanelsSize = panel_off(kNT);
static_assert(kPanelsSize == kNTiles * kTile * kTile, "the panels hold the lower tiles exactly");
// entry (r, c) of the panels; r >= 6 floor(c / 6)
__device__ __forceinline__ int pix(int r, int c) {
    const int kt = c / kTile;
    return panel_off(kt) + (c - kTile * kt) * (kBlk - kTile * kt) + (r - kTile * kt);
}

template <class T>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};
// six consecutive entries from shared memory (p is 8-byte aligned for float,
// 16-byte for double: every tile starts at an even index)
template <class T>
__device__ __forceinline__ void lds6(const T* p, T v[kTile]) {
    using V = typename Vec2<T>::type;
    const V* q = reinterpret_cast<const V*>(p);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const V w = q[i];
        v[2 * i] = w.x;
        v[2 * i + 1] = w.y;
    }
}
// s_r x s_c as FP32 with x FP64: x rounded by f64_to_f32_rn, then scaled in
// FP32; x outside 2^+-100 is scaled in FP64 before rounding, so an entry
// beyond the FP32 range still maps to its finite scaled value. 9,216 FP64
// scalings per block were the FP32 inversion's largest single cost.
__device__ __forceinline__ float scaled_f32(double x, float sr, float sc) {
    float f;
    if (f64_to_f32_rn(x, f)) return f * (sr * sc);
    // |x| < 2^-100 with s_r s_c <= 2^70: the scaled entry is below 2^-30,
    // under FP32 resolution beside the unit diagonal, so it is 0 (near the
    // rest state such residues of cancelling FP32 Hessian terms are common
    // and would each take the FP64 path)
    const unsigned ex = (unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu;
    if (ex < 1023u - 100u && sr * sc <= 0x1p70f) return 0.f;
    return (float)(x * (double)sr * (double)sc);
}
__device__ __forceinline__ float inv_sqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double inv_sqrt(double x) { return 1.0 / sqrt(x); }
// non-negative floats and doubles order like their bit patterns
__device__ __forceinline__ void smem_max(float* p, float v) {
    atomicMax(reinterpret_cast<unsigned*>(p), __float_as_uint(v));
}
__device__ __forceinline__ void smem_max(double* p, double v) {
    atomicMax(reinterpret_cast<unsigned long long*>(p), (unsigned long long)__double_as_longlong(v));
}

// The block's inverse B = s W^T W s is kept as W' = W diag(s) (B = W'^T W'),
// packed by 4-row-aligned columns (wcol): warp w writes columns w, w +
// nwarps, ... with its lanes on consecutive rows (coalesced), from W in
// shared memory (kPanels: the packed column panels, pix; otherwise W^T,
// wt[c * 96 + r] = W[r][c]); the rows of a column's first quad above the
// diagonal are written as zeros. Storing the factor instead of B halves the
// bytes of every later apply, needs no W^T W product here, and keeps B
// positive semi-definite whatever the rounding of W'.
template <bool kPanels>
__device__ __forceinline__ int wix(int r, int c) {
    if constexpr (kPanels)
        return pix(r, c);
    else
        return c * kBlk + r;
}
template <class R, class T, bool kPanels = false>
__device__ __forceinline__ void store_factor(const Dev<R>& D, int b, const T* wt, const T* sc) {
    if (D.blocks16) {
        // BF16 tiles (IPC_PREC_BF16_MAS): tile (i, j) row-major, written in
        // order so the global stores coalesce (the column reads of W^T take
        // bank conflicts: a one-time cost per restart)
        __nv_bfloat16* d16 = static_cast<__nv_bfloat16*>(D.blocks16) + (size_t)b * kW16;
        for (int e = threadIdx.x; e < kW16; e += blockDim.x) {
            const int tix = e >> 8;
            int ti = 0;
            while ((ti + 1) * (ti + 2) / 2 <= tix) ++ti;
            const int tj = tix - ti * (ti + 1) / 2;
            const int r = kT16 * ti + ((e >> 4) & 15), c = kT16 * tj + (e & 15);
            d16[e] = __float2bfloat16_rn(r >= c ? (float)(wt[wix<kPanels>(r, c)] * sc[c]) : 0.f);
        }
        return;
    }
    R* dst = D.blocks + (size_t)b * kW;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int j = warp; j < kBlk; j += nw) {
        const T s = sc[j];
        const int r0 = j & ~3;
        R* out = dst + wcol(j) - r0;
        for (int r = r0 + lane; r < kBlk; r += 32) out[r] = r >= j ? (R)(wt[wix<kPanels>(r, j)] * s) : (R)0;
    }
}

// Blocks come from the FP64 assembly (level 0: asmb, coarse levels: asmbc);
// only entries at or below a block's diagonal are read (level 0 holds no
// others).
// flags: pass 0 (T = float) marks a block whose factorisation floored or
// raised a pivot, i.e. whose conditioning FP32 cannot carry (very stiff
// contacts, coarse aggregates); pass 1 (T = double) re-inverts only the
// marked blocks. flags == nullptr: no marks.
template <class R, class T>
__global__ void __launch_bounds__(kInvThreads) k_invert(Dev<R> D, int* flags, int pass) {
    extern __shared__ unsigned char smem_raw[];
    T* buf = reinterpret_cast<T*>(smem_raw);      // 96 x 96: L^T, then W
    T* vec = buf + kBlk * kBlk;                   // 2 x 96 broadcast
    T* sc = vec + 2 * kBlk;                       // diagonal scaling s
    T* idg = sc + kBlk;                           // 1 / L_kk
    T* pm = idg + kBlk;                           // 3 rotating slots: max_r L_rk^2 of step k
    __shared__ int s_bad;
    const T eps_piv = (T)(sizeof(T) == 8 ? 1e-12 : 1e-6);
    int b = blockIdx.x;
    if (pass == 1 && !flags[b]) return;  // uniform over the CTA
    int l = 0;
    while (l + 1 < D.nlev && b >= D.blk_off[l + 1]) ++l;
    int grp = b - D.blk_off[l];
    const int* mem = D.members[l] + (size_t)grp * kSub;
    const double* src = l == 0 ? D.asmb + (size_t)b * kBlk * kBlk
                               : D.asmbc + (size_t)(b - D.blk_off[1]) * kBlk * kBlk;
    if (threadIdx.x == 0) {
        s_bad = 0;
        pm[0] = pm[1] = pm[2] = (T)0;
    }
    for (int r = threadIdx.x; r < kBlk; r += blockDim.x) {
        double d = src[r * kBlk + r];
        sc[r] = (mem[r / 3] < 0 || !(d > 0.0)) ? (T)1 : (T)(1.0 / sqrt(d));
    }
    // Cholesky: thread t owns tile (ti, tj), ti >= tj, the tiles ordered by
    // column from the right (column 15, then 14, ...), so that the tiles still
    // active at panel kt (columns >= kt) are the first (16 - kt)(17 - kt) / 2
    // threads and the warps past them skip the panel's work
    const int t = threadIdx.x;
    const bool act = t < kNTiles;
    int ti = 0, tj = 0;
    if (act) {
        int rem = t, c = kNT - 1;
        while (rem >= kNT - c) {
            rem -= kNT - c;
            --c;
        }
        tj = c;
        ti = c + rem;
    }
    int r0 = kTile * ti, c0 = kTile * tj;
    __syncthreads();
    T a[kTile][kTile];
#pragma unroll
    for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
        for (int cc = 0; cc < kTile; ++cc) {
            int r = r0 + rr, c = c0 + cc;
            T v = (T)0;
            if (act) {
                if (mem[r / 3] < 0 || mem[c / 3] < 0)
                    v = (r == c) ? (T)1 : (T)0;
                else if constexpr (sizeof(T) == 4)
                    v = scaled_f32(src[r * kBlk + c], sc[r], sc[c]);
                else
                    v = (T)(src[r * kBlk + c] * (double)sc[r] * (double)sc[c]);
            }
            a[rr][cc] = v;
        }

    // ---- S = L L^T (lower tiles in registers)
    for (int kt = 0; kt < kNT; ++kt) {
#pragma unroll
        for (int kk = 0; kk < kTile; ++kk) {
            const int k = kTile * kt + kk;
            T* vb = vec + (k & 1) * kBlk;
            T* pmk = pm + k % 3;
            // slot (k + 1) % 3 was last read in step k - 2, which every thread
            // finished before the previous barrier; step k + 1 writes it after
            // the next one
            if (threadIdx.x == 0) pm[(k + 1) % 3] = (T)0;
            if (act && tj == kt) {
                T m = (T)0;
#pragma unroll
                for (int rr = 0; rr < kTile; ++rr) {
                    T v = (ti == kt && rr < kk) ? (T)0 : a[rr][kk];
                    vb[r0 + rr] = v;
                    if ((ti > kt || rr > kk) && v * v > m) m = v * v;
                }
                if (m > (T)0) smem_max(pmk, m);
            }
            __syncthreads();
            if (act && ti >= kt && tj >= kt) {
                // pivot floor, then the row-norm bound L_rk^2 <= S_rr = 1 that
                // holds for any SPD matrix: where rounding breaks it the pivot
                // is raised (a diagonal shift, as in a modified Cholesky), so
                // L stays bounded and no floored pivot can cascade
                const T raw = vb[k];
                T piv = raw;
                if (!(piv > eps_piv)) piv = eps_piv;
                const T pmax = *pmk;
                if (pmax > piv) piv = pmax;
                if (ti == kt && tj == kt && piv != raw) s_bad = 1;
                // L_kk = piv * isq, the column below scaled by isq, the trailing
                // update by ip = isq^2: L L^T reproduces the rank-1 update exactly
                // up to the rounding of isq
                const T isq = inv_sqrt(piv);
                const T sq = piv * isq, ip = isq * isq;
                if (ti == kt && tj == kt) idg[k] = isq;
                T vr[kTile], vc[kTile];
                lds6(vb + r0, vr);
                lds6(vb + c0, vc);
#pragma unroll
                for (int q = 0; q < kTile; ++q) vc[q] *= ip;
#pragma unroll
                for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
                    for (int cc = 0; cc < kTile; ++cc) {
                        if (tj == kt && cc < kk) continue;    // finished columns
                        if (tj == kt && cc == kk) {
                            // column k of L
                            if (ti > kt || rr > kk) a[rr][cc] = vr[rr] * isq;
                            else if (rr == kk) a[rr][cc] = sq;
                        } else {
                            a[rr][cc] -= vr[rr] * vc[cc];
                        }
                    }
            }
        }
    }
    // L^T -> shared memory (lower entries only; nothing reads above the diagonal)
#pragma unroll
    for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
        for (int cc = 0; cc < kTile; ++cc)
            if (act && (ti > tj || rr >= cc)) buf[(c0 + cc) * kBlk + r0 + rr] = a[rr][cc];
    __syncthreads();

    // W = L^{-1}: tiles in row order, t = ti (ti + 1) / 2 + tj
    if (act) {
        int rem = t;
        ti = 0;
        while (rem > ti) {
            ++ti;
            rem -= ti;
        }
        tj = rem;
    }
    r0 = kTile * ti;
    c0 = kTile * tj;
    // ---- W = L^{-1}: row k of W is final once divided by L_kk; then every
    // later row r subtracts L_rk times it
#pragma unroll
    for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
        for (int cc = 0; cc < kTile; ++cc) a[rr][cc] = (act && ti == tj && rr == cc) ? (T)1 : (T)0;
    for (int kt = 0; kt < kNT; ++kt) {
#pragma unroll
        for (int kk = 0; kk < kTile; ++kk) {
            const int k = kTile * kt + kk;
            T* vb = vec + (k & 1) * kBlk;
            const T* Lk = buf + k * kBlk;                 // column k of L
            if (act && ti == kt) {
                const T il = idg[k];
#pragma unroll
                for (int cc = 0; cc < kTile; ++cc) {
                    a[kk][cc] *= il;
                    vb[c0 + cc] = a[kk][cc];
                }
            }
            __syncthreads();
            if (act && ti >= kt && tj <= kt) {
                T lr[kTile], wc[kTile];
                lds6(Lk + r0, lr);
                lds6(vb + c0, wc);
#pragma unroll
                for (int q = 0; q < kTile; ++q)
                    if (!(ti > kt || q > kk)) lr[q] = (T)0;
#pragma unroll
                for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
                    for (int cc = 0; cc < kTile; ++cc) a[rr][cc] -= lr[rr] * wc[cc];
            }
        }
    }
    __syncthreads();
    // W^T -> shared memory (buf[c * 96 + r] = W[r][c], r >= c): column j of W
    // is then contiguous for the packed store below
#pragma unroll
    for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
        for (int cc = 0; cc < kTile; ++cc)
            if (act && (ti > tj || rr >= cc)) buf[(c0 + cc) * kBlk + r0 + rr] = a[rr][cc];
    if (pass == 0 && flags && threadIdx.x == 0) flags[b] = s_bad;
    // the final factorisation of this block (FP64 form, or the FP64 redo)
    // modified a pivot: counted for the parity checks
    if ((pass == 1 || !flags) && threadIdx.x == 0 && s_bad && D.pivfix) atomicAdd(D.pivfix, 1);
    __syncthreads();
    store_factor<R, T>(D, b, buf, sc);
}

// FP32 first pass of the block inversion, blocked by the same 6x6 tiles: per
// panel of 6 columns, the diagonal tile's thread factors its tile in
// registers, the tiles below solve against it (L_ik = A_ik L_kk^-T), and every
// trailing tile takes the rank-6 update A_ij -= L_ik L_jk^T from a shared
// panel buffer; W = L^-1 follows by tile rows the same way. Two barriers per
// panel and one per W row block replace one per column, and the updates are
// runs of 36 FMAs on operands from shared memory. The pivot rules of k_invert
// are not reproduced here: a block whose factorisation would floor a pivot
// or raise one (some L_rk^2 > 1) is flagged and returned early, and the FP64
// pass inverts it with those rules; every other block is an unmodified
// Cholesky factorisation, which is what k_invert computes for it too.
template <class R>
__global__ void __launch_bounds__(kInvThreads, 6) k_invert_tiled(Dev<R> D, int* flags) {
    static_assert(sizeof(R) == 4, "FP32 first pass");
    extern __shared__ unsigned char smem_raw[];
    float* buf = reinterpret_cast<float*>(smem_raw);  // packed column panels (pix): A, then L, then W
    float* pan = buf + kPanelsSize;                    // 2 x 6 x 96: panel columns of L, then row blocks of W
    float* sc = pan + 2 * kTile * kBlk;                // diagonal scaling s
    float* idg = sc + kBlk;                            // 1 / L_kk
    __shared__ int s_bad;
    const float eps_piv = D.piv32;
    const int b = blockIdx.x;
    int l = 0;
    while (l + 1 < D.nlev && b >= D.blk_off[l + 1]) ++l;
    const int grp = b - D.blk_off[l];
    const int* mem = D.members[l] + (size_t)grp * kSub;
    const double* src = l == 0 ? D.asmb + (size_t)b * kBlk * kBlk
                               : D.asmbc + (size_t)(b - D.blk_off[1]) * kBlk * kBlk;
    __shared__ unsigned char pad[kBlk];  // padded slot (no node)
    if (threadIdx.x == 0) s_bad = 0;
    for (int r = threadIdx.x; r < kBlk; r += blockDim.x) {
        const double d = src[r * kBlk + r];
        const bool pr = mem[r / 3] < 0;
        pad[r] = pr ? 1 : 0;
        sc[r] = (pr || !(d > 0.0)) ? 1.f : (float)(1.0 / sqrt(d));
    }
    __syncthreads();
    // the scaled block staged in buf (row-major), a warp per row and a lane
    // per column so the FP64 reads coalesce; 4 rows per pass keep 12
    // independent loads in flight per lane. Entries above the diagonal inside
    // the diagonal 6 x 6 tiles are zero; padded slots carry an identity.
    {
        constexpr int kRows = 4;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        for (int r0 = warp * kRows; r0 < kBlk; r0 += nw * kRows) {
            double v[kRows][3];
#pragma unroll
            for (int q = 0; q < kRows; ++q)
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const int r = r0 + q, c = lane + 32 * m;
                    v[q][m] = (r < kBlk && c <= r) ? src[r * kBlk + c] : 0.0;
                }
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                const int r = r0 + q;
                if (r >= kBlk) break;
                const int cend = (r / kTile + 1) * kTile;
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const int c = lane + 32 * m;
                    if (c >= cend) continue;
                    float f;
                    if (c > r)
                        f = 0.f;
                    else if (pad[r] || pad[c])
                        f = (r == c) ? 1.f : 0.f;
                    else
                        f = scaled_f32(v[q][m], sc[r], sc[c]);
                    buf[pix(r, c)] = f;
                }
            }
        }
    }
    // Cholesky: tiles ordered by column from the right, as in k_invert
    const int t = threadIdx.x;
    const bool act = t < kNTiles;
    int ti = 0, tj = 0;
    if (act) {
        int rem = t, c = kNT - 1;
        while (rem >= kNT - c) {
            rem -= kNT - c;
            --c;
        }
        tj = c;
        ti = c + rem;
    }
    int r0 = kTile * ti, c0 = kTile * tj;
    // the thread's tile in the panels: column cc at tb + cc * ld, 6 rows each
    int tb = panel_off(tj) + (r0 - c0), ld = kBlk - c0;
    __syncthreads();
    float a[kTile][kTile];
#pragma unroll
    for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
        for (int cc = 0; cc < kTile; ++cc) a[rr][cc] = act ? buf[tb + cc * ld + rr] : 0.f;
    __syncthreads();  // buf is reused for L^T below
    bool bad = false;
    for (int kt = 0; kt < kNT; ++kt) {
        float* P = pan + (kt & 1) * (kTile * kBlk);  // P[m * 96 + row] = L[row][6 kt + m]
        if (act && ti == kt && tj == kt) {
#pragma unroll
            for (int c = 0; c < kTile; ++c) {
                float piv = a[c][c];
                if (!(piv > eps_piv)) {
                    piv = eps_piv;
                    bad = true;
                }
                const float isq = rsqrtf(piv);
                a[c][c] = piv * isq;
                idg[kTile * kt + c] = isq;
#pragma unroll
                for (int r = c + 1; r < kTile; ++r) {
                    a[r][c] *= isq;
                    if (!(a[r][c] * a[r][c] <= 1.f)) bad = true;  // NaN too
                }
#pragma unroll
                for (int r = c + 1; r < kTile; ++r)
#pragma unroll
                    for (int q = c + 1; q <= r; ++q) a[r][q] -= a[r][c] * a[q][c];
            }
#pragma unroll
            for (int m = 0; m < kTile; ++m)
#pragma unroll
                for (int r = 0; r < kTile; ++r) P[m * kBlk + r0 + r] = (r >= m) ? a[r][m] : 0.f;
        }
        __syncthreads();
        if (act && ti > kt && tj == kt) {
            float Lk[kTile][kTile], il[kTile];  // L_kk (strictly lower part used) and 1 / diag
#pragma unroll
            for (int c = 0; c < kTile; ++c) {
                il[c] = idg[kTile * kt + c];
#pragma unroll
                for (int m = 0; m < c; ++m) Lk[c][m] = P[m * kBlk + kTile * kt + c];
            }
#pragma unroll
            for (int c = 0; c < kTile; ++c)
#pragma unroll
                for (int r = 0; r < kTile; ++r) {
                    float x = a[r][c];
#pragma unroll
                    for (int m = 0; m < c; ++m) x -= a[r][m] * Lk[c][m];
                    x *= il[c];
                    a[r][c] = x;
                    if (!(x * x <= 1.f)) bad = true;
                }
#pragma unroll
            for (int m = 0; m < kTile; ++m)
#pragma unroll
                for (int r = 0; r < kTile; ++r) P[m * kBlk + r0 + r] = a[r][m];
        }
        __syncthreads();
        if (act && tj > kt) {
#pragma unroll
            for (int m = 0; m < kTile; ++m) {
                float vr[kTile], vc[kTile];
                lds6(P + m * kBlk + r0, vr);
                lds6(P + m * kBlk + c0, vc);
#pragma unroll
                for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
                    for (int cc = 0; cc < kTile; ++cc) a[rr][cc] -= vr[rr] * vc[cc];
            }
        }
    }
    if (bad) s_bad = 1;
    // L -> the panels, in place of A (lower entries only)
#pragma unroll
    for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
        for (int cc = 0; cc < kTile; ++cc)
            if (act && (ti > tj || rr >= cc)) buf[tb + cc * ld + rr] = a[rr][cc];
    __syncthreads();
    if (s_bad) {  // uniform over the CTA: the FP64 pass inverts this block
        if (threadIdx.x == 0) flags[b] = 1;
        return;
    }

    // W = L^-1 by tile rows, tiles in row order: at step kt, row block kt is
    // solved against L_kk; every later row block subtracts L_i,kt W_kt,j
    if (act) {
        int rem = t;
        ti = 0;
        while (rem > ti) {
            ++ti;
            rem -= ti;
        }
        tj = rem;
    }
    r0 = kTile * ti;
    c0 = kTile * tj;
    tb = panel_off(tj) + (r0 - c0);
    ld = kBlk - c0;
#pragma unroll
    for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
        for (int cc = 0; cc < kTile; ++cc) a[rr][cc] = (act && ti == tj && rr == cc) ? 1.f : 0.f;
    for (int kt = 0; kt < kNT; ++kt) {
        float* Q = pan + (kt & 1) * (kTile * kBlk);  // Q[m * 96 + col] = W[6 kt + m][col]
        if (act && ti == kt) {
            const int k0 = kTile * kt;
#pragma unroll
            for (int r = 0; r < kTile; ++r) {
                float Lr[kTile];
#pragma unroll
                for (int m = 0; m < r; ++m) Lr[m] = buf[panel_off(kt) + m * (kBlk - k0) + r];
                const float ir = idg[k0 + r];
#pragma unroll
                for (int cc = 0; cc < kTile; ++cc) {
                    float x = a[r][cc];
#pragma unroll
                    for (int m = 0; m < r; ++m) x -= Lr[m] * a[m][cc];
                    a[r][cc] = x * ir;
                }
            }
#pragma unroll
            for (int m = 0; m < kTile; ++m)
#pragma unroll
                for (int cc = 0; cc < kTile; ++cc) Q[m * kBlk + c0 + cc] = a[m][cc];
        }
        __syncthreads();
        if (act && ti > kt && tj <= kt) {
#pragma unroll
            for (int m = 0; m < kTile; ++m) {
                float lr[kTile], wc[kTile];
                lds6(buf + panel_off(kt) + m * (kBlk - kTile * kt) + (r0 - kTile * kt), lr);
                lds6(Q + m * kBlk + c0, wc);
#pragma unroll
                for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
                    for (int cc = 0; cc < kTile; ++cc) a[rr][cc] -= lr[rr] * wc[cc];
            }
        }
    }
    __syncthreads();
    // W -> the panels, in place of L (every thread has finished reading L)
#pragma unroll
    for (int rr = 0; rr < kTile; ++rr)
#pragma unroll
        for (int cc = 0; cc < kTile; ++cc)
            if (act && (ti > tj || rr >= cc)) buf[tb + cc * ld + rr] = a[rr][cc];
    if (threadIdx.x == 0) flags[b] = 0;
    __syncthreads();
    store_factor<R, float, true>(D, b, buf, sc);
}

// ------------------------------------------------------ C_base snapshot

template <class R>
__global__ void k_snapshot(Dev<R> D) {
    int n = min(*D.C.count, D.cap);
    if (blockIdx.x == 0 && threadIdx.x == 0) *D.Cb.count = n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        D.Cb.type[i] = D.C.type[i];
        D.Cb.v[i] = D.C.v[i];
        unsigned long long key = D.C.key[i];
        D.Cb.key[i] = key;
        D.Cb.d[i] = D.C.d[i];
        D.Cb.k[i] = D.C.k[i];
        D.Cb.bp[i] = D.C.bp[i];
        for (int r = 0; r < 3; ++r) D.Cb.r[3 * i + r] = D.C.r[3 * i + r];
        for (int r = 0; r < 4; ++r) D.Cb.w[4 * i + r] = D.C.w[4 * i + r];
        unsigned h = (unsigned)(mix64(key) & (unsigned long long)(D.btab - 1));
        for (int probe = 0; probe < D.btab; ++probe) {
            unsigned long long old = atomicCAS(&D.bkeys[h], ~0ULL, key);
            if (old == ~0ULL || old == key) {
                D.bidx[h] = i;
                break;
            }
            h = (h + 1) & (D.btab - 1);
        }
    }
}

// ------------------------------------------------------ classification

template <class R>
__device__ __forceinline__ int base_lookup(const Dev<R>& D, unsigned long long key) {
    unsigned h = (unsigned)(mix64(key) & (unsigned long long)(D.btab - 1));
    for (int probe = 0; probe < D.btab; ++probe) {
        unsigned long long k = D.bkeys[h];
        if (k == key) return D.bidx[h];
        if (k == ~0ULL) return -1;
        h = (h + 1) & (D.btab - 1);
    }
    return -1;
}

template <class R>
__global__ void k_classify(Dev<R> D, ContactBuf C) {
    int n = min(*C.count, D.cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double k = C.k[i];
        int b = base_lookup(D, C.key[i]);
        double dS;
        if (b < 0) {
            dS = k;
        } else {
            double ww = 0, wb = 0, bb = 0;
            for (int j = 0; j < 4; ++j) {
                ww += C.w[4 * i + j] * C.w[4 * i + j];
                wb += C.w[4 * i + j] * D.Cb.w[4 * b + j];
                bb += D.Cb.w[4 * b + j] * D.Cb.w[4 * b + j];
            }
            double rr = C.r[3 * i] * D.Cb.r[3 * b] + C.r[3 * i + 1] * D.Cb.r[3 * b + 1] + C.r[3 * i + 2] * D.Cb.r[3 * b + 2];
            double cosang = wb * rr / sqrt(ww * bb);
            double kb = D.Cb.k[b];
            if (cosang < D.cos_rot)
                dS = k;
            else if (k > kb)
                dS = k - kb;
            else
                dS = 0.0;
        }
        if (!(dS > 0.0)) continue;
        int u = atomicAdd(&D.S->n_upd, 1);
        if (u >= D.upd_cap) {
            atomicOr(&D.S->overflow, 4);
            continue;
        }
        D.upd_c[u] = i;
        D.upd_dS[u] = dS;
        int4 q = C.v[i];
        int vid[4] = {q.x, q.y, q.z, q.w};
        int nvv = C.type[i] == 2 ? 1 : 4;
        int gs[4];
        for (int j = 0; j < nvv; ++j) {
            int g = D.grp0[vid[j]];
            bool dup = false;
            for (int m = 0; m < j; ++m) dup |= gs[m] == g;
            gs[j] = dup ? -1 : g;
            if (!dup) atomicAdd(&D.upd_cnt[g], 1);
        }
    }
}

template <class R>
__global__ void k_fill_lists(Dev<R> D, ContactBuf C) {
    int n = min(D.S->n_upd, D.upd_cap);
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        int i = D.upd_c[u];
        int4 q = C.v[i];
        int vid[4] = {q.x, q.y, q.z, q.w};
        int nvv = C.type[i] == 2 ? 1 : 4;
        int gs[4];
        for (int j = 0; j < nvv; ++j) {
            int g = D.grp0[vid[j]];
            bool dup = false;
            for (int m = 0; m < j; ++m) dup |= gs[m] == g;
            gs[j] = dup ? -1 : g;
            if (!dup) D.upd_list[D.upd_off[g] + atomicAdd(&D.upd_cur[g], 1)] = u;
        }
    }
}

// one warp per subdomain: K rounds of "best entry ranked below the last pick"
template <class R>
__global__ void k_topk(Dev<R> D, ContactBuf C) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= D.ngroups[0]) return;
    int beg = D.upd_off[warp], end = D.upd_off[warp + 1];
    double lastS = __longlong_as_double(0x7ff0000000000000ULL);
    unsigned long long lastK = 0;
    bool have_last = false;
    for (int r = 0; r < D.K; ++r) {
        double bestS = -1.0;
        unsigned long long bestK = ~0ULL;
        int bestU = -1;
        for (int e = beg + lane; e < end; e += 32) {
            int u = D.upd_list[e];
            double s = D.upd_dS[u];
            unsigned long long k = C.key[D.upd_c[u]];
            // strictly below the last pick in (dS desc, key asc) order
            if (have_last && !(s < lastS || (s == lastS && k > lastK))) continue;
            if (s > bestS || (s == bestS && k < bestK)) {
                bestS = s;
                bestK = k;
                bestU = u;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            double s2 = __shfl_xor_sync(0xffffffffu, bestS, o);
            unsigned long long k2 = __shfl_xor_sync(0xffffffffu, bestK, o);
            int u2 = __shfl_xor_sync(0xffffffffu, bestU, o);
            if (s2 > bestS || (s2 == bestS && k2 < bestK)) {
                bestS = s2;
                bestK = k2;
                bestU = u2;
            }
        }
        if (lane == 0) D.topk[(size_t)warp * D.K + r] = bestU;
        if (bestU < 0) {
            for (int r2 = r + 1 + lane; r2 < D.K; r2 += 32) D.topk[(size_t)warp * D.K + r2] = -1;
            break;
        }
        lastS = bestS;
        lastK = bestK;
        have_last = true;
    }
}

// ------------------------------------------------------ preconditioner apply

// r_{l+1}[g] = sum of the level-l values over the members of level-l
// subdomain g (C_{l+1} sums xyz per cluster): one warp per subdomain, lane =
// slot, no atomics
template <class R>
__global__ void k_restrict_level(Dev<R> D, int l, const R* __restrict__ src) {
    int grp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (grp >= D.ngroups[l]) return;
    int node = D.members[l][(size_t)grp * kSub + lane];
    R a0 = 0, a1 = 0, a2 = 0;
    if (node >= 0) {
        a0 = src[3 * node];
        a1 = src[3 * node + 1];
        a2 = src[3 * node + 2];
    }
    a0 = warp_sum(a0);
    a1 = warp_sum(a1);
    a2 = warp_sum(a2);
    if (lane == 0) {
        R* dst = D.coarse_r + D.coarse_off[l + 1] + 3 * grp;
        dst[0] = a0;
        dst[1] = a1;
        dst[2] = a2;
    }
}

// Shared by both block applies: wait (bounded) for the block's factor; a
// wait that runs out records the timeout in the scene's status, drains the
// copy still in flight and makes the whole CTA leave (z stays unwritten).
template <class R>
__device__ __forceinline__ bool factor_arrived(const Dev<R>& D, uint64_t* bar) {
    const bool arrived = mbar_wait(bar, 0, D.wait_polls);
    if (__syncthreads_or(!arrived)) {
        if (threadIdx.x == 0) {
            D.S->async_timeout = 1;
            mbar_wait(bar, 0, kDrainPolls);
        }
        return false;
    }
    return true;
}

// four consecutive values from shared memory (16-byte aligned for float,
// two 16-byte loads for double)
template <class R>
__device__ __forceinline__ void ld4(const R* p, R v[4]) {
    if constexpr (sizeof(R) == 4) {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else {
        const double2 a = reinterpret_cast<const double2*>(p)[0], c = reinterpret_cast<const double2*>(p)[1];
        v[0] = a.x;
        v[1] = a.y;
        v[2] = c.x;
        v[3] = c.y;
    }
}
template <class R>
__device__ __forceinline__ void st4(R* p, const R v[4]) {
    if constexpr (sizeof(R) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
}

// Y = W' X for NC columns X[a] (96 values each, shared memory) with the
// packed factor in shared memory; 96 threads. Warp w, lane 8k + q owns row
// quad i = 8w + q (rows 4i..4i+3) and the column chunk [24k, 24k + 24): at
// each step the 8 lanes of a load phase read consecutive quads of one column
// (no bank conflicts) and the columns above row 4i + 3 are skipped; the four
// chunks' partial sums meet by shuffles.
template <class R, int NC>
__device__ __forceinline__ void lower_apply(const R* __restrict__ Ws, const R (*X)[kBlk], R (*Y)[kBlk], int nc) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = lane & 7, k = lane >> 3;
    const int i = 8 * warp + q;
    R acc[NC][4];
#pragma unroll
    for (int a = 0; a < NC; ++a)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[a][r] = 0;
    const int j0 = 24 * k, jend = min(j0 + 24, 4 * i + 4);
    for (int j = j0; j < jend; ++j) {
        R w[4];
        ld4(Ws + wcol(j) + 4 * i - (j & ~3), w);
#pragma unroll
        for (int a = 0; a < NC; ++a) {
            if (a >= nc) break;
            const R xj = X[a][j];
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[a][r] += w[r] * xj;
        }
    }
#pragma unroll
    for (int a = 0; a < NC; ++a) {
        if (a >= nc) break;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            acc[a][r] += __shfl_xor_sync(0xffffffffu, acc[a][r], 8);
            acc[a][r] += __shfl_xor_sync(0xffffffffu, acc[a][r], 16);
        }
        if (k == 0) st4(&Y[a][4 * i], acc[a]);
    }
}

// z = W'^T y (y in shared memory, z into shared memory); 96 threads. Each
// round a warp takes four columns, 8 lanes per column: lane k of a column
// handles the row quads k, k + 8, k + 16 (its quads of y stay in registers)
// and the 8 lanes read consecutive quads of the column; a 3-step shuffle sums
// them.
template <class R>
__device__ __forceinline__ void upper_apply(const R* __restrict__ Ws, const R* __restrict__ y, R* __restrict__ z) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cl = lane >> 3, k = lane & 7;
    R yq[3][4];
#pragma unroll
    for (int m = 0; m < 3; ++m) ld4(y + 4 * (k + 8 * m), yq[m]);
#pragma unroll 2
    for (int round = 0; round < 8; ++round) {
        const int c = 4 * (3 * round + warp) + cl;
        const int a = c >> 2;
        const R* col = Ws + wcol(c) - 4 * a;
        R acc = 0;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const int Q = k + 8 * m;
            if (Q >= a) {
                R w[4];
                ld4(col + 4 * Q, w);
                acc += w[0] * yq[m][0] + w[1] * yq[m][1] + w[2] * yq[m][2] + w[3] * yq[m][3];
            }
        }
        acc += __shfl_xor_sync(0xffffffffu, acc, 1);
        acc += __shfl_xor_sync(0xffffffffu, acc, 2);
        acc += __shfl_xor_sync(0xffffffffu, acc, 4);
        if (k == 0) z[c] = acc;
    }
}

// The right-hand side entry of thread tid for block b: its node (< 0 for a
// padded slot) and value; level 0 reads g, coarse levels their restricted
// residuals. Two dependent global loads, issued one block ahead by the
// persistent applies so their latency overlaps the current block's products.
template <class R>
__device__ __forceinline__ void gather_rhs(const Dev<R>& D, const R* __restrict__ g, int b, int tid, int& l, int& node,
                                           R& val) {
    l = 0;
    while (l + 1 < D.nlev && b >= D.blk_off[l + 1]) ++l;
    const int grp = b - D.blk_off[l];
    node = D.members[l][(size_t)grp * kSub + tid / 3];
    const int comp = tid % 3;
    if (node < 0)
        val = (R)0;
    else
        val = l == 0 ? g[3 * node + comp] : D.coarse_r[D.coarse_off[l] + 3 * node + comp];
}

// Block apply without Woodbury updates (restart iterations, coarse levels):
// z_b = B_b r_b = W'^T (W' r_b), 96 threads per CTA. The CTAs are persistent
// (a few per SM) and stream their blocks through a 2-stage ring in shared
// memory: each packed factor (19.2 KB in FP32) arrives as one bulk copy
// (cp.async.bulk, completing on its slot's mbarrier) issued two blocks ahead,
// so the copies of later blocks overlap the gathers and products of the
// current one and no CTA waits out a partial last wave.
constexpr int kApplyCtasPerSm = 5;

template <class R>
__global__ void __launch_bounds__(96) k_block_apply_plain(Dev<R> D, const R* __restrict__ g, R* __restrict__ z) {
    extern __shared__ __align__(128) unsigned char bsm[];  // 2 slots of kW values
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ __align__(16) R rhs[kBlk];
    __shared__ __align__(16) R ys[kBlk];
    constexpr uint32_t kBytes = kW * sizeof(R);
    const int nb = D.blk_off[D.nlev];
    const int tid = threadIdx.x;
    const int first = blockIdx.x, stride = gridDim.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        for (int s = 0; s < 2; ++s) {
            const int b = first + s * stride;
            if (b < nb) {
                mbar_arrive_expect_tx(&bar[s], kBytes);
                bulk_g2s(bsm + s * kBytes, D.blocks + (size_t)b * kW, kBytes, &bar[s]);
            }
        }
    }
    int it = 0;
    int l_n = 0, node_n = -1;
    R val_n = (R)0;
    if (first < nb) gather_rhs(D, g, first, tid, l_n, node_n, val_n);
    for (int b = first; b < nb; b += stride, ++it) {
        const int slot = it & 1;
        const uint32_t parity = (uint32_t)(it >> 1) & 1u;
        const R* Ws = reinterpret_cast<const R*>(bsm + slot * kBytes);
        const int l = l_n, node = node_n, comp = tid % 3;
        rhs[tid] = val_n;
        if (b + stride < nb) gather_rhs(D, g, b + stride, tid, l_n, node_n, val_n);  // next block's, in flight
        __syncthreads();  // rhs complete; the barriers' initialisation is visible
        const bool arrived = mbar_wait(&bar[slot], parity, D.wait_polls);
        if (__syncthreads_or(!arrived)) {
            // record, drain the copies still in flight (this slot's and the
            // other slot's, if one was issued), leave z unwritten
            if (tid == 0) {
                D.S->async_timeout = 1;
                mbar_wait(&bar[slot], parity, kDrainPolls);
                if (b + stride < nb) mbar_wait(&bar[slot ^ 1], (uint32_t)((it + 1) >> 1) & 1u, kDrainPolls);
            }
            return;
        }
        lower_apply<R, 1>(Ws, &rhs, &ys, 1);
        __syncthreads();
        upper_apply(Ws, ys, rhs);  // rhs is free: z into it
        __syncthreads();           // every read of this slot and of ys is done
        const R out = rhs[tid];
        if (tid == 0 && b + 2 * stride < nb) {
            // reuse the slot: order the generic reads above before the copy
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[slot], kBytes);
            bulk_g2s(bsm + slot * kBytes, D.blocks + (size_t)(b + 2 * stride) * kW, kBytes, &bar[slot]);
        }
        if (node >= 0) {
            if (l == 0)
                z[3 * node + comp] = out;
            else
                D.coarse_y[D.coarse_off[l] + 3 * node + comp] = out;
        }
        const double od = (double)out;
        if (!(od - od == 0.0)) atomicCAS(&D.S->dbg_block, -1, b);
        __syncthreads();  // rhs is rewritten by the next block
    }
}

// ---- BF16 factors on the tensor cores (IPC_PREC_BF16_MAS)
//
// W' is stored as BF16 16 x 16 tiles. y = W' x and z = W'^T y run as
// mma.sync m16n8k16 (BF16 operands, FP32 accumulation) with A the factor
// tiles loaded by ldmatrix (.trans for W'^T) and B the right-hand sides, each
// split into a BF16 high part and a BF16 low part (x - hi) in two columns of
// the 8 so that only the factor carries BF16 rounding: y = D[:, 0] + D[:, 1].
// B = W'^T W' stays symmetric positive semi-definite whatever the rounding.

__device__ __forceinline__ int tile16(int i, int j) { return i * (i + 1) / 2 + j; }

__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_k, hi_k);  // .x = first (lower k)
    return *reinterpret_cast<const uint32_t*>(&v);
}
// high and low BF16 parts of two consecutive values, as two packed registers
__device__ __forceinline__ void split_bf16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat16 ah = __float2bfloat16_rn(a), bh = __float2bfloat16_rn(b);
    const __nv_bfloat162 h2 = __halves2bfloat162(ah, bh);
    hi = *reinterpret_cast<const uint32_t*>(&h2);
    lo = pack_bf16(a - __bfloat162float(ah), b - __bfloat162float(bh));
}
__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// A fragment of tile T (16 x 16 BF16, row-major, 32-byte rows): lane L points
// at row (L & 7) + 8 ((L >> 3) & 1), column 8 (L >> 4); for T^T the 8 x 8
// quarters swap: row (L & 7) + 8 (L >> 4), column 8 ((L >> 3) & 1)
__device__ __forceinline__ void frag_tile(uint32_t a[4], const __nv_bfloat16* T, bool transposed) {
    const int L = threadIdx.x & 31;
    if (!transposed)
        ldsm_x4(a, T + ((L & 7) + 8 * ((L >> 3) & 1)) * kT16 + 8 * (L >> 4));
    else
        ldsm_x4_t(a, T + ((L & 7) + 8 * (L >> 4)) * kT16 + 8 * ((L >> 3) & 1));
}
// B fragment of one 16-row segment x of a right-hand side: column 0 its high
// parts, column 1 its low parts, the other columns zero (lanes with g >= 2)
__device__ __forceinline__ void frag_rhs(const float* x, uint32_t& b0, uint32_t& b1) {
    const int L = threadIdx.x & 31, g = L >> 2, t = L & 3;
    b0 = b1 = 0u;
    if (g < 2) {
        uint32_t h0, l0, h1, l1;
        split_bf16x2(x[2 * t], x[2 * t + 1], h0, l0);
        split_bf16x2(x[2 * t + 8], x[2 * t + 9], h1, l1);
        b0 = g == 0 ? h0 : l0;
        b1 = g == 0 ? h1 : l1;
    }
}

// y = W' x (trans = false) or y = W'^T x (trans = true) for one vector, 96
// threads: warp w takes the output tiles w and 5 - w (equal work)
__device__ __forceinline__ void tri_apply_bf16(const __nv_bfloat16* Wt, const float* x, float* y, bool trans) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int o = u == 0 ? warp : kNT16 - 1 - warp;  // output tile
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        const int k0 = trans ? o : 0, k1 = trans ? kNT16 - 1 : o;
        for (int k = k0; k <= k1; ++k) {
            uint32_t a[4], b0, b1;
            // y_o += W'_ok x_k (k <= o), or y_o += W'_ko^T x_k (k >= o)
            frag_tile(a, Wt + (size_t)(trans ? tile16(k, o) : tile16(o, k)) * (kT16 * kT16), trans);
            frag_rhs(x + kT16 * k, b0, b1);
            mma_bf16(acc, a, b0, b1);
        }
        if (t == 0) {
            y[kT16 * o + g] = acc[0] + acc[1];
            y[kT16 * o + g + 8] = acc[2] + acc[3];
        }
    }
}

// V[a] = W' X[a] for a < nc (nc <= 1 + kMaxK) right-hand sides in shared
// memory: their high and low parts fill 2 nc columns, 8 per mma; warp w
// takes the row tiles w and 5 - w. The pair of columns (2a, 2a + 1) lands in
// lane t = a % 4 of n-tile a / 4.
__device__ __forceinline__ void lower_apply_bf16(const __nv_bfloat16* Wt, const float (*X)[kBlk], float (*V)[kBlk],
                                                 int nc) {
    constexpr int kNq = (2 * (1 + kMaxK) + 7) / 8;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int nq = (2 * nc + 7) / 8;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int o = u == 0 ? warp : kNT16 - 1 - warp;
        float acc[kNq][4];
#pragma unroll
        for (int q = 0; q < kNq; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = 0.f;
        for (int k = 0; k <= o; ++k) {
            uint32_t a[4];
            frag_tile(a, Wt + (size_t)tile16(o, k) * (kT16 * kT16), false);
#pragma unroll
            for (int q = 0; q < kNq; ++q) {
                if (q >= nq) break;
                const int n = 8 * q + g, col = n >> 1;
                uint32_t b0 = 0u, b1 = 0u;
                if (col < nc) {
                    const float* x = X[col] + kT16 * k;
                    uint32_t h0, l0, h1, l1;
                    split_bf16x2(x[2 * t], x[2 * t + 1], h0, l0);
                    split_bf16x2(x[2 * t + 8], x[2 * t + 9], h1, l1);
                    b0 = (n & 1) ? l0 : h0;
                    b1 = (n & 1) ? l1 : h1;
                }
                mma_bf16(acc[q], a, b0, b1);
            }
        }
#pragma unroll
        for (int q = 0; q < kNq; ++q) {
            const int col = 4 * q + t;
            if (q < nq && col < nc) {
                V[col][kT16 * o + g] = acc[q][0] + acc[q][1];
                V[col][kT16 * o + g + 8] = acc[q][2] + acc[q][3];
            }
        }
    }
}

// Plain block apply with BF16 factors: the persistent 2-stage ring of
// k_block_apply_plain with 10.7 KB tiles and the two products on the tensor
// cores.
__global__ void __launch_bounds__(96) k_block_apply_plain16(Dev<float> D, const float* __restrict__ g,
                                                            float* __restrict__ z) {
    extern __shared__ __align__(128) unsigned char bsm[];  // 2 slots of kW16 BF16 values
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ __align__(16) float rhs[kBlk];
    __shared__ __align__(16) float ys[kBlk];
    constexpr uint32_t kBytes = kW16 * 2;
    const __nv_bfloat16* src16 = static_cast<const __nv_bfloat16*>(D.blocks16);
    const int nb = D.blk_off[D.nlev];
    const int tid = threadIdx.x;
    const int first = blockIdx.x, stride = gridDim.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        for (int s = 0; s < 2; ++s) {
            const int b = first + s * stride;
            if (b < nb) {
                mbar_arrive_expect_tx(&bar[s], kBytes);
                bulk_g2s(bsm + s * kBytes, src16 + (size_t)b * kW16, kBytes, &bar[s]);
            }
        }
    }
    int it = 0;
    int l_n = 0, node_n = -1;
    float val_n = 0.f;
    if (first < nb) gather_rhs(D, g, first, tid, l_n, node_n, val_n);
    for (int b = first; b < nb; b += stride, ++it) {
        const int slot = it & 1;
        const uint32_t parity = (uint32_t)(it >> 1) & 1u;
        const __nv_bfloat16* Wt = reinterpret_cast<const __nv_bfloat16*>(bsm + slot * kBytes);
        const int l = l_n, node = node_n, comp = tid % 3;
        rhs[tid] = val_n;
        if (b + stride < nb) gather_rhs(D, g, b + stride, tid, l_n, node_n, val_n);  // next block's, in flight
        __syncthreads();
        const bool arrived = mbar_wait(&bar[slot], parity, D.wait_polls);
        if (__syncthreads_or(!arrived)) {
            if (tid == 0) {
                D.S->async_timeout = 1;
                mbar_wait(&bar[slot], parity, kDrainPolls);
                if (b + stride < nb) mbar_wait(&bar[slot ^ 1], (uint32_t)((it + 1) >> 1) & 1u, kDrainPolls);
            }
            return;
        }
        tri_apply_bf16(Wt, rhs, ys, false);
        __syncthreads();
        tri_apply_bf16(Wt, ys, rhs, true);  // z into rhs
        __syncthreads();
        const float out = rhs[tid];
        if (tid == 0 && b + 2 * stride < nb) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(&bar[slot], kBytes);
            bulk_g2s(bsm + slot * kBytes, src16 + (size_t)(b + 2 * stride) * kW16, kBytes, &bar[slot]);
        }
        if (node >= 0) {
            if (l == 0)
                z[3 * node + comp] = out;
            else
                D.coarse_y[D.coarse_off[l] + 3 * node + comp] = out;
        }
        if (!(out - out == 0.f)) atomicCAS(&D.S->dbg_block, -1, b);
        __syncthreads();
    }
}

// Level-0 apply with the Sparse-Input Woodbury update (Eq. 7) and the plain
// apply of the coarse blocks. With U_d the subdomain's top-K vectors (ns of
// them) and V = W' [g_d, U_d]:
//   C = I + V_U^T V_U = I + U^T B U,  r = V_U^T V_g = U^T B g,
//   C lambda = r (FP64 Cholesky, one warp, a lane per row),
//   z_d = W'^T (V_g - V_U lambda) = B g - B U lambda.
// One pass of the factor over all 1 + ns columns and one transposed pass.
template <class R, bool kB16 = false>
__global__ void __launch_bounds__(96) k_block_apply(Dev<R> D, const R* __restrict__ g, R* __restrict__ z,
                                                    ContactBuf C, int woodbury) {
    static_assert(!kB16 || sizeof(R) == 4, "BF16 factors come with the FP32 bulk");
    extern __shared__ __align__(128) unsigned char wsm[];  // the packed factor (bulk copy)
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(16) R rhs[1 + kMaxK][kBlk];
    __shared__ __align__(16) R V[1 + kMaxK][kBlk];
    __shared__ __align__(16) R zs[kBlk];
    __shared__ double cap[kMaxK][kMaxK + 1];  // C, then its factor; column kMaxK: r
    __shared__ double rr[kMaxK];
    __shared__ double lam[kMaxK];
    __shared__ double qb_sh;
    __shared__ int keep;
    __shared__ int sel[kMaxK];
    __shared__ int nsel;
    const R* Ws = reinterpret_cast<const R*>(wsm);
    const __nv_bfloat16* Wt = reinterpret_cast<const __nv_bfloat16*>(wsm);
    const int b = blockIdx.x;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        constexpr uint32_t kBytes = kB16 ? kW16 * 2 : kW * sizeof(R);
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, kBytes);
        if constexpr (kB16)
            bulk_g2s(wsm, static_cast<const __nv_bfloat16*>(D.blocks16) + (size_t)b * kW16, kBytes, &bar);
        else
            bulk_g2s(wsm, D.blocks + (size_t)b * kW, kBytes, &bar);
    }
    int l = 0;
    while (l + 1 < D.nlev && b >= D.blk_off[l + 1]) ++l;
    const int grp = b - D.blk_off[l];
    const int* mem = D.members[l] + (size_t)grp * kSub;
    const int node = mem[tid / 3];
    const int comp = tid % 3;
    if (l == 0)
        rhs[0][tid] = node >= 0 ? g[3 * node + comp] : (R)0;
    else
        rhs[0][tid] = node >= 0 ? D.coarse_r[D.coarse_off[l] + 3 * node + comp] : (R)0;
    if (tid == 0) {
        int n = 0;
        if (l == 0 && woodbury)
            for (int a = 0; a < D.K; ++a) {
                const int u = D.topk[(size_t)grp * D.K + a];
                if (u < 0) break;
                sel[n++] = u;
            }
        nsel = n;
    }
    __syncthreads();
    const int ns = nsel;
    for (int a = 0; a < ns; ++a) rhs[1 + a][tid] = (R)0;
    __syncthreads();
    if (tid < ns) {  // column tid of U_d: u = sqrt(dS) w_j r at the slot of vertex j
        const int u = sel[tid];
        const int i = D.upd_c[u];
        const double sq = sqrt(D.upd_dS[u]);
        const int4 q = C.v[i];
        const int vid[4] = {q.x, q.y, q.z, q.w};
        const int nvv = C.type[i] == 2 ? 1 : 4;
        for (int j = 0; j < nvv; ++j) {
            if (D.grp0[vid[j]] != grp) continue;
            const int s = D.slot0[vid[j]];
            const double wj = sq * C.w[4 * i + j];
            for (int r = 0; r < 3; ++r) rhs[1 + tid][3 * s + r] += (R)(wj * C.r[3 * i + r]);
        }
    }
    __syncthreads();
    if (!factor_arrived(D, &bar)) return;
    // V = W' [rhs]: one read of each factor entry for all 1 + ns columns
    if constexpr (kB16)
        lower_apply_bf16(Wt, rhs, V, 1 + ns);
    else if (ns == 0)
        lower_apply<R, 1>(Ws, rhs, V, 1);
    else
        lower_apply<R, 1 + kMaxK>(Ws, rhs, V, 1 + ns);
    __syncthreads();
    if (ns > 0) {
        // C = I + V_U^T V_U (the half a <= c), r = V_U^T V_g and |V_g|^2: dot
        // products of bulk-precision vectors summed in R per warp, the warp
        // totals in FP64 (FP64 products would add no accuracy to FP32 values,
        // and this GPU runs FP64 at a small fraction of its FP32 rate)
        const int nsym = ns * (ns + 1) / 2;
        for (int e = warp; e < nsym + ns + 1; e += 3) {
            const R* va;
            const R* vb;
            int a = -1, c = -1;
            if (e < nsym) {
                a = 0;
                int rem = e;
                while (rem >= ns - a) {
                    rem -= ns - a;
                    ++a;
                }
                c = a + rem;
                va = V[1 + a];
                vb = V[1 + c];
            } else if (e < nsym + ns) {
                a = e - nsym;
                va = V[1 + a];
                vb = V[0];
            } else {
                va = V[0];
                vb = V[0];
            }
            R sacc = 0;
            for (int i = lane; i < kBlk; i += 32) sacc += va[i] * vb[i];
            sacc = warp_sum(sacc);
            if (lane == 0) {
                if (c >= 0) {
                    cap[a][c] = (double)sacc + (a == c ? 1.0 : 0.0);
                    cap[c][a] = cap[a][c];
                } else if (a >= 0) {
                    rr[a] = (double)sacc;
                } else {
                    qb_sh = (double)sacc;
                }
            }
        }
        __syncthreads();
        if (warp == 0) {
            // Cholesky of the SPD capacitance system by one warp, lane i holding
            // row i: per column one reciprocal square root and a trailing
            // update of the rows below. C = I + U^T B U >= I in exact
            // arithmetic, so every pivot is >= 1; a pivot below 1/2 means B's
            // rounding swamped a stiff update direction, and the correction is
            // dropped (z_d = B g_d)
            bool good = true;
            for (int j = 0; j < ns; ++j) {
                const double d = cap[j][j];
                good = good && (d >= 0.5);
                const double il = rsqrt(fmax(d, 0.5));
                __syncwarp();
                if (lane > j && lane < ns) cap[lane][j] *= il;
                __syncwarp();
                if (lane > j && lane < ns) {
                    const double lij = cap[lane][j];
                    for (int k = j + 1; k <= lane; ++k) cap[lane][k] -= lij * cap[k][j];
                }
                if (lane == j) cap[j][j] = il;  // 1 / L_jj
                __syncwarp();
            }
            // L y = r, then L^T lambda = y: lane i keeps the running value of
            // row i; each step broadcasts one solved entry
            double t = lane < ns ? rr[lane] : 0.0;
            for (int j = 0; j < ns; ++j) {
                const double yj = __shfl_sync(0xffffffffu, t * cap[j < 32 ? j : 0][j], j);
                if (lane == j) t = yj;
                if (lane > j && lane < ns) t -= cap[lane][j] * yj;
            }
            for (int j = ns - 1; j >= 0; --j) {
                const double lj = __shfl_sync(0xffffffffu, t * cap[j][j], j);
                if (lane == j) t = lj;
                if (lane < j) t -= cap[j][lane] * lj;
            }
            // g^T B~ g = |V_g|^2 - r^T lambda must lie in [0, g^T B g]
            // (adding U U^T only lowers the quadratic form); outside that range
            // (FP32 factors of stiff blocks make the solve unstable), or with a
            // non-finite lambda, the correction is dropped
            double rl = lane < ns ? rr[lane] * t : 0.0;
            bool fin = lane < ns ? (t - t == 0.0) : true;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rl += __shfl_xor_sync(0xffffffffu, rl, o);
            fin = __all_sync(0xffffffffu, fin);
            const double qb = qb_sh, qc = qb - rl;
            const bool ok = good && fin && qc <= qb * (1.0 + 1e-3) && qc >= -1e-3 * qb;
            if (lane < ns) lam[lane] = ok ? t : 0.0;
            if (lane == 0) keep = ok;
        }
        __syncthreads();
        double o = (double)V[0][tid];
        if (keep)
            for (int a = 0; a < ns; ++a) o -= lam[a] * (double)V[1 + a][tid];
        __syncthreads();
        V[0][tid] = (R)o;
    }
    __syncthreads();
    if constexpr (kB16)
        tri_apply_bf16(Wt, V[0], zs, true);
    else
        upper_apply(Ws, V[0], zs);
    __syncthreads();
    const R out = zs[tid];
    if (node >= 0) {
        if (l == 0)
            z[3 * node + comp] = out;
        else
            D.coarse_y[D.coarse_off[l] + 3 * node + comp] = out;
    }
    // diagnostics: record the first block whose output is not finite
    const double od = (double)out;
    if (!(od - od == 0.0) && atomicCAS(&D.S->dbg_block, -1, b) == -1) D.S->dbg_ns = ns;
}

template <class R>
__global__ void k_prolong(Dev<R> D, R* __restrict__ z) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= D.nv) return;
    R a0 = z[3 * v], a1 = z[3 * v + 1], a2 = z[3 * v + 2];
    for (int l = 1; l < D.nlev; ++l) {
        const R* y = D.coarse_y + D.coarse_off[l] + 3 * D.node_of_vert[l][v];
        a0 += y[0];
        a1 += y[1];
        a2 += y[2];
    }
    z[3 * v] = a0;
    z[3 * v + 1] = a1;
    z[3 * v + 2] = a2;
}

template <class R>
__global__ void k_clear_upd(Dev<R> D) {
    D.S->n_upd = 0;
}

// ---- 3x3 block-Jacobi preconditioner (the paper's MAS-vs-Jacobi ablation,
// Sec. 5.1): P = blockdiag(H_vv)^-1 over the vertices, H_vv the 3x3 diagonal
// blocks of H_base at the restart, read from the level-0 assembly (lower
// triangle) and inverted in FP64 by cofactors.
template <class R>
__global__ void k_jacobi_build(Dev<R> D) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= D.nv) return;
    const double* A = D.asmb + (size_t)D.grp0[v] * (kBlk * kBlk) + (size_t)(3 * D.slot0[v]) * kBlk + 3 * D.slot0[v];
    const double a = A[0], b = A[kBlk], c = A[2 * kBlk], d = A[kBlk + 1], e = A[2 * kBlk + 1], f = A[2 * kBlk + 2];
    // symmetric [[a b c] [b d e] [c e f]]
    const double c00 = d * f - e * e, c01 = c * e - b * f, c02 = b * e - c * d;
    const double c11 = a * f - c * c, c12 = b * c - a * e, c22 = a * d - b * b;
    const double det = a * c00 + b * c01 + c * c02;
    const double id = det > 0.0 ? 1.0 / det : 0.0;
    R* J = D.jac + 9 * (size_t)v;
    const double m[9] = {c00, c01, c02, c01, c11, c12, c02, c12, c22};
#pragma unroll
    for (int k = 0; k < 9; ++k) J[k] = (R)(m[k] * id);
}

template <class R>
__global__ void k_jacobi_apply(Dev<R> D, const R* __restrict__ g, R* __restrict__ z) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= D.nv) return;
    const R* J = D.jac + 9 * (size_t)v;
    const R g0 = g[3 * v], g1 = g[3 * v + 1], g2 = g[3 * v + 2];
#pragma unroll
    for (int r = 0; r < 3; ++r) z[3 * v + r] = J[3 * r] * g0 + J[3 * r + 1] * g1 + J[3 * r + 2] * g2;
}

}  // namespace

template <class R>
void launch_restart(const Dev<R>& D, const double* x, const ContactBuf& C, cudaStream_t st) {
    int nb = D.blk_off[D.nlev];
    KL(k_clear_upd<R><<<1, 1, 0, st>>>(D));
    if (D.pivfix) cudaMemsetAsync(D.pivfix, 0, sizeof(int), st);
    const int nb0 = D.nlev > 1 ? D.blk_off[1] : nb;
    KL(k_init_blocks<R><<<nblk((long long)nb * (kBlk * kBlk / 4), 256), 256, 0, st>>>(D, nb0, nb));
    KL(k_tet_hessian<R><<<nblk(D.nt, 64), 64, 0, st>>>(D, x));
    KL(k_assemble_tets0<R><<<nblk(D.nt), kT, 0, st>>>(D));
    if (D.nitem > 0) {
        KL(k_asm_contrib<R><<<nblk(D.nt), kT, 0, st>>>(D));
        KL(k_asm_sum<R><<<nblk(32LL * D.nitem, 256), 256, 0, st>>>(D));
    }
    const int ncn = D.coarse_off[D.nlev] / 3;
    if (ncn > 0) cudaMemsetAsync(D.pg_k, 0, sizeof(double) * ncn, st);
    KL(k_assemble_contacts<R><<<592, kT, 0, st>>>(D, C));
    if (ncn > 0) KL(k_assemble_pg_coarse<R><<<nblk(ncn), kT, 0, st>>>(D));
    if (D.jac)
        KL(k_jacobi_build<R><<<nblk(D.nv), kT, 0, st>>>(D));
    else
        launch_invert(D, st);
    cudaMemsetAsync(D.bkeys, 0xFF, sizeof(unsigned long long) * D.btab, st);
    KL(k_snapshot<R><<<592, kT, 0, st>>>(D));
}

template <class R>
void launch_invert(const Dev<R>& D, cudaStream_t st) {
    const int nb = D.blk_off[D.nlev];
    // blocks are assembled in FP64 and inverted in the bulk precision R (FP32
    // in the mixed mode: B300's FP64 rate, about two FMAs per clock per SM,
    // would make the inversion the most expensive step) with an FP64 redo of
    // the blocks FP32 cannot carry
    const size_t smem_r = sizeof(R) * ((size_t)kBlk * kBlk + 4 * kBlk + 4);
    const size_t smem_d = sizeof(double) * ((size_t)kBlk * kBlk + 4 * kBlk + 4);
    const size_t smem_t = sizeof(float) * ((size_t)kPanelsSize + 2 * kTile * kBlk + 2 * kBlk);
    static const bool attr_set = [&] {  // once per process, thread-safe
        cudaFuncSetAttribute(k_invert<R, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_r);
        cudaFuncSetAttribute(k_invert<R, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_d);
        if (sizeof(R) == 4)
            cudaFuncSetAttribute(k_invert_tiled<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_t);
        return true;
    }();
    (void)attr_set;
    if (sizeof(R) == 4) {
        // FP32 first; the blocks that floored or raised a pivot again in FP64
        if constexpr (sizeof(R) == 4) KL(k_invert_tiled<R><<<nb, kInvThreads, smem_t, st>>>(D, D.invflag));
        KL(k_invert<R, double><<<nb, kInvThreads, smem_d, st>>>(D, D.invflag, 1));
    } else {
        KL(k_invert<R, R><<<nb, kInvThreads, smem_r, st>>>(D, nullptr, 0));
    }
}

template <class R>
void launch_classify(const Dev<R>& D, const ContactBuf& C, cudaStream_t st) {
    int ng = D.ngroups[0];
    KL(k_clear_upd<R><<<1, 1, 0, st>>>(D));
    cudaMemsetAsync(D.upd_cnt, 0, sizeof(int) * ng, st);
    cudaMemsetAsync(D.upd_cur, 0, sizeof(int) * ng, st);
    KL(k_classify<R><<<592, kT, 0, st>>>(D, C));
    scan_exclusive(D.upd_cnt, D.upd_off, ng, D.gtmp, st);
    KL(k_fill_lists<R><<<592, kT, 0, st>>>(D, C));
    KL(k_topk<R><<<nblk(32LL * ng), kT, 0, st>>>(D, C));
}

template <class R>
void launch_restrict(const Dev<R>& D, const R* g, cudaStream_t st) {
    if (D.jac) return;  // block-Jacobi: no coarse levels
    for (int l = 0; l + 1 < D.nlev; ++l) {
        const R* src = l == 0 ? g : D.coarse_r + D.coarse_off[l];
        KL(k_restrict_level<R><<<nblk(32LL * D.ngroups[l]), kT, 0, st>>>(D, l, src));
    }
}

template <class R>
void launch_blocks(const Dev<R>& D, const R* g, R* z, const ContactBuf& C, bool woodbury, cudaStream_t st) {
    static const int sms = [] {  // once per process, thread-safe
        cudaFuncSetAttribute(k_block_apply_plain<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(2 * kW * sizeof(R)));
        cudaFuncSetAttribute(k_block_apply<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(kW * sizeof(R)));
        if constexpr (sizeof(R) == 4) {
            cudaFuncSetAttribute(k_block_apply_plain16, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kW16 * 2);
            cudaFuncSetAttribute(k_block_apply<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kW16 * 2);
        }
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 148;
    }();
    const int nb = D.blk_off[D.nlev];
    if (D.jac) {
        KL(k_jacobi_apply<R><<<nblk(D.nv), kT, 0, st>>>(D, g, z));
        return;
    }
    if constexpr (sizeof(R) == 4) {
        if (D.blocks16) {
            // BF16 factors: tiles of 10.7 KB, more persistent CTAs per SM
            if (woodbury)
                KL(k_block_apply<R, true><<<nb, 96, kW16 * 2, st>>>(D, g, z, C, 1));
            else
                KL(k_block_apply_plain16<<<std::min(nb, (D.apply_ctas > 0 ? D.apply_ctas : 8) * sms), 96,
                                           2 * kW16 * 2, st>>>(D, g, z));
            return;
        }
    }
    if (woodbury) {
        KL(k_block_apply<R><<<nb, 96, kW * sizeof(R), st>>>(D, g, z, C, 1));
    } else {
        // persistent CTAs: as many as fit at once (two FP64 rings per SM, five
        // FP32), never more than the blocks
        const int per_sm = D.apply_ctas > 0 ? D.apply_ctas : (sizeof(R) == 8 ? 2 : kApplyCtasPerSm);
        KL(k_block_apply_plain<R><<<std::min(nb, per_sm * sms), 96, 2 * kW * sizeof(R), st>>>(D, g, z));
    }
}

template <class R>
int autotune_apply(Dev<R>& D, cudaStream_t st) {
    // candidate CTAs per SM of the persistent plain apply, bounded by its
    // 2-slot ring in shared memory: FP64 factors 38.4 KB a slot, FP32 19.2
    // KB, BF16 10.7 KB
    std::vector<int> cand;
    if (sizeof(R) == 8)
        cand = {1, 2};
    else if (D.blocks16)
        cand = {4, 6, 8, 10};
    else
        cand = {2, 3, 4, 5};
    if (D.jac || D.blk_off[D.nlev] < 2 * 148) return D.apply_ctas = cand.back();  // small scenes: one block a CTA
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return D.apply_ctas = 0;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return D.apply_ctas = 0;
    }
    // zero factors and gradient: the timing does not depend on the values
    const int nb = D.blk_off[D.nlev];
    if (D.blocks16)
        cudaMemsetAsync(D.blocks16, 0, (size_t)nb * kW16 * 2, st);
    else
        cudaMemsetAsync(D.blocks, 0, (size_t)nb * kW * sizeof(R), st);
    cudaMemsetAsync(D.g, 0, sizeof(R) * 3 * (size_t)D.nv, st);
    if (D.nlev > 1) cudaMemsetAsync(D.coarse_r, 0, sizeof(R) * (size_t)D.coarse_off[D.nlev], st);
    int best = 0;
    float best_ms = 0.f;
    constexpr int kReps = 8;
    for (int c : cand) {
        D.apply_ctas = c;
        launch_blocks(D, D.g, D.z, D.C, false, st);  // warm
        cudaEventRecord(a, st);
        for (int r = 0; r < kReps; ++r) launch_blocks(D, D.g, D.z, D.C, false, st);
        cudaEventRecord(b, st);
        float ms = 0.f;
        if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
            best = 0;
            break;
        }
        if (best == 0 || ms < best_ms) {
            best = c;
            best_ms = ms;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return D.apply_ctas = best;
}

template <class R>
void launch_prolong(const Dev<R>& D, R* z, cudaStream_t st) {
    if (D.nlev > 1 && !D.jac) KL(k_prolong<R><<<nblk(D.nv), kT, 0, st>>>(D, z));
}

template <class R>
void launch_precond(const Dev<R>& D, const R* g, R* z, const ContactBuf& C, bool woodbury, cudaStream_t st) {
    launch_restrict(D, g, st);
    launch_blocks(D, g, z, C, woodbury, st);
    launch_prolong(D, z, st);
}

#define INST(R)                                                                                            \
    template void launch_restart<R>(const Dev<R>&, const double*, const ContactBuf&, cudaStream_t);         \
    template void launch_invert<R>(const Dev<R>&, cudaStream_t);                                          \
    template int autotune_apply<R>(Dev<R>&, cudaStream_t);                                                \
    template void launch_classify<R>(const Dev<R>&, const ContactBuf&, cudaStream_t);                     \
    template void launch_precond<R>(const Dev<R>&, const R*, R*, const ContactBuf&, bool, cudaStream_t);   \
    template void launch_restrict<R>(const Dev<R>&, const R*, cudaStream_t);                              \
    template void launch_blocks<R>(const Dev<R>&, const R*, R*, const ContactBuf&, bool, cudaStream_t);    \
    template void launch_prolong<R>(const Dev<R>&, R*, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace ipcb
