// Incremental potential (Eq. 1) and its gradient: inertia, stable neo-Hookean
// elasticity and the IPC barrier; the predictor; trial positions; prefix scan.
//
// Elastic energy density (reading of the SNH the paper cites):
//   Psi(F) = mu/2 (|F|^2 - 3) - mu (J - 1) + lambda/2 (J - 1)^2,
//   P = mu F + (lambda (J - 1) - mu) cof(F),  F = Ds B,  grad_{x_j} = V P B^T e_j.
// Energies are accumulated in FP64; gradients in R. With an FP32 bulk the
// elastic energy is formed in double-float arithmetic (about 48 significant
// bits) on the FP32 pipes: the FP64 pipe of this GPU is a small fraction of
// its FP32 rate and was the bound of the all-FP64 form.
#include "kernels.h"

namespace ipcb {

namespace {

constexpr int kT = 256;

inline int nblk(long long n, int t = kT) { return (int)((n + t - 1) / t); }

template <class R>
__global__ void k_predict(Dev<R> D) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * D.nv) return;
    int r = i % 3;
    double x = D.x[i];
    D.xs[i] = x;
    D.xt[i] = x + D.h * D.v[i] + D.h * D.h * D.gravity[r];
}

template <class R>
__global__ void k_trial(Dev<R> D, int mode, double c) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * D.nv) return;
    if (mode == 0) {
        // when the per-subdomain verification fell back to the uniform step
        // and the per-body one did not, the first trial is the per-body step
        // (verified, and no smaller anywhere than the uniform one)
        const Scalars* S = D.S;
        if (S->ccd_passes < 0 && S->ccd_passes_b >= 0 && S->alpha_bmax > S->alpha_min) {
            mode = 1;
            c = 1.0;
        }
    }
    double a = mode == 0 ? D.alpha[D.grp0[i / 3]] : (mode == 1 ? c * D.alpha_b[D.body[i / 3]] : c);
    D.xtry[i] = D.x[i] + a * (double)D.p[i];
}

// Double-float values (Dekker, "A floating-point technique for extending the
// available precision", 1971; Knuth, TAOCP vol. 2, Sec. 4.2.2): an unevaluated
// sum hi + lo of two floats with |lo| <= ulp(hi) / 2. two_sum and two_prod
// are error-free; df_add is the short form whose error is a few units of
// 2^-47 times the larger operand, which is the size of the inputs' own
// representation error here. The _rn intrinsics are never fused into an FMA,
// which the error-free steps rely on.
struct df {
    float hi, lo;
};
__device__ __forceinline__ df fast_two_sum(float a, float b) {  // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df df_add(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, {-b.hi, -b.lo}); }
__device__ __forceinline__ df df_mul(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);  // exact residual of the product
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ df df_mulf(df a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return fast_two_sum(p, e);
}
__device__ __forceinline__ double df_val(df a) { return (double)a.hi + (double)a.lo; }

// g = M (x - x~), E += 1/2 (x - x~)^T M (x - x~). With an FP32 bulk it also
// stores x as float hi / lo parts for the elastic pass that follows.
template <class R>
__global__ void k_inertia(Dev<R> D, const double* __restrict__ x, R* __restrict__ g, double* E) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (v < D.nv) {
        if constexpr (sizeof(R) == 4) {
            float hi[3], lo[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                const double xv = x[3 * v + r];
                hi[r] = (float)xv;
                lo[r] = (float)(xv - (double)hi[r]);  // xv - hi is exact
            }
            D.xsplit[2 * (size_t)v] = make_float4(hi[0], hi[1], hi[2], 0.f);
            D.xsplit[2 * (size_t)v + 1] = make_float4(lo[0], lo[1], lo[2], 0.f);
        }
        double m = D.massd[v];
        double d0 = x[3 * v] - D.xt[3 * v];
        double d1 = x[3 * v + 1] - D.xt[3 * v + 1];
        double d2 = x[3 * v + 2] - D.xt[3 * v + 2];
        e = 0.5 * m * (d0 * d0 + d1 * d1 + d2 * d2);
        if (g) {
            g[3 * v] = (R)(m * d0);
            g[3 * v + 1] = (R)(m * d1);
            g[3 * v + 2] = (R)(m * d2);
        }
    }
    warp_add_to(E, e);
}

template <class R>
__device__ __forceinline__ void load_B(const Dev<R>& D, int t, double B[3][3]) {
    const R* base = D.tetB + (size_t)(t / kPack) * 9 * kPack + (t % kPack);
#pragma unroll
    for (int c = 0; c < 9; ++c) B[c / 3][c % 3] = (double)base[c * kPack];
}

// Elastic energy and gradient with an FP32 bulk: Ds, F, |F|^2, J and the
// energy in double-float from the hi / lo positions k_inertia stored (B is
// exact in FP32; the coefficients h^2 V mu / 2, h^2 V mu, h^2 V lam / 2 are
// float pairs), summed per warp in double-float and added to E in FP64 once
// per warp; the gradient in FP32 from F's leading floats.
__global__ void k_elastic_df(Dev<float> D, float* __restrict__ g, double* E) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    df e = {0.f, 0.f};
    if (t < D.nt) {
        const int4 q = D.tets[t];
        const int vid[4] = {q.x, q.y, q.z, q.w};
        df X[4][3];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 h = D.xsplit[2 * (size_t)vid[j]], l = D.xsplit[2 * (size_t)vid[j] + 1];
            X[j][0] = {h.x, l.x};
            X[j][1] = {h.y, l.y};
            X[j][2] = {h.z, l.z};
        }
        float B[3][3];
        const float* base = D.tetB + (size_t)(t / kPack) * 9 * kPack + (t % kPack);
#pragma unroll
        for (int c = 0; c < 9; ++c) B[c / 3][c % 3] = base[c * kPack];
        df Ds[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int j = 0; j < 3; ++j) Ds[r][j] = df_sub(X[j + 1][r], X[0][r]);
        df F[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c)
                F[r][c] = df_add(df_add(df_mulf(Ds[r][0], B[0][c]), df_mulf(Ds[r][1], B[1][c])),
                                 df_mulf(Ds[r][2], B[2][c]));
        const df C00 = df_sub(df_mul(F[1][1], F[2][2]), df_mul(F[2][1], F[1][2]));
        const df C01 = df_sub(df_mul(F[2][1], F[0][2]), df_mul(F[0][1], F[2][2]));
        const df C02 = df_sub(df_mul(F[0][1], F[1][2]), df_mul(F[1][1], F[0][2]));
        const df J = df_add(df_add(df_mul(F[0][0], C00), df_mul(F[1][0], C01)), df_mul(F[2][0], C02));
        df Ic = {-3.f, 0.f};
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Ic = df_add(Ic, df_mul(F[r][c], F[r][c]));
        const df Jm1 = df_add(J, {-1.f, 0.f});
        const float2 e0 = D.tet_ec[3 * (size_t)t], e1 = D.tet_ec[3 * (size_t)t + 1], e2 = D.tet_ec[3 * (size_t)t + 2];
        const df ca = {e0.x, e0.y}, cb = {e1.x, e1.y}, cc = {e2.x, e2.y};
        // h^2 V (mu/2 (|F|^2 - 3) - mu (J - 1) + lam/2 (J - 1)^2)
        e = df_add(df_sub(df_mul(ca, Ic), df_mul(cb, Jm1)), df_mul(df_mul(cc, Jm1), Jm1));
        if (g) {
            // h^2 V P = cb F + (2 cc (J - 1) - cb) cof(F)
            const float s = 2.f * cc.hi * Jm1.hi - cb.hi;
            float Fr[3][3], Cr[3][3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) Fr[r][c] = F[r][c].hi;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int a = (c + 1) % 3, b = (c + 2) % 3;
                Cr[0][c] = Fr[1][a] * Fr[2][b] - Fr[2][a] * Fr[1][b];
                Cr[1][c] = Fr[2][a] * Fr[0][b] - Fr[0][a] * Fr[2][b];
                Cr[2][c] = Fr[0][a] * Fr[1][b] - Fr[1][a] * Fr[0][b];
            }
            float Pm[3][3], G[3][3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) Pm[r][c] = cb.hi * Fr[r][c] + s * Cr[r][c];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float acc = 0.f;
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc += Pm[r][c] * B[j][c];
                    G[r][j] = acc;
                }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                atomicAdd(&g[3 * vid[0] + r], -(G[r][0] + G[r][1] + G[r][2]));
#pragma unroll
                for (int j = 0; j < 3; ++j) atomicAdd(&g[3 * vid[j + 1] + r], G[r][j]);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        e = df_add(e, {__shfl_xor_sync(0xffffffffu, e.hi, o), __shfl_xor_sync(0xffffffffu, e.lo, o)});
    if ((threadIdx.x & 31) == 0 && e.hi != 0.f) atomicAdd(E, df_val(e));
}

template <class R>
__global__ void k_elastic(Dev<R> D, const double* __restrict__ x, R* __restrict__ g, double* E) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    if (t < D.nt) {
        int4 q = D.tets[t];
        int vid[4] = {q.x, q.y, q.z, q.w};
        double X[4][3];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 3; ++r) X[j][r] = x[3 * vid[j] + r];
        double B[3][3];
        load_B(D, t, B);
        double F[3][3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double s = 0.0;
#pragma unroll
                for (int j = 0; j < 3; ++j) s += (X[j + 1][r] - X[0][r]) * B[j][c];
                F[r][c] = s;
            }
        // J = f0 . (f1 x f2): the first cofactor column in FP64 (the energy
        // check needs J - 1 to FP64 accuracy); the gradient's cofactors are
        // formed in R below
        const double C0[3] = {F[1][1] * F[2][2] - F[2][1] * F[1][2], F[2][1] * F[0][2] - F[0][1] * F[2][2],
                              F[0][1] * F[1][2] - F[1][1] * F[0][2]};
        double J = F[0][0] * C0[0] + F[1][0] * C0[1] + F[2][0] * C0[2];
        double Ic = 0.0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int c = 0; c < 3; ++c) Ic += F[r][c] * F[r][c];
        double mu = D.tet_mu[t], lam = D.tet_lam[t], V = D.tet_vol[t];
        double h2V = D.h * D.h * V;
        e = h2V * (0.5 * mu * (Ic - 3.0) - mu * (J - 1.0) + 0.5 * lam * (J - 1.0) * (J - 1.0));
        if (g) {
            R s = (R)(lam * (J - 1.0) - mu);
            R Fr[3][3], Cr[3][3];  // F and its cofactor matrix (columns f_a x f_b) in R
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) Fr[r][c] = (R)F[r][c];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int a = (c + 1) % 3, b = (c + 2) % 3;
                Cr[0][c] = Fr[1][a] * Fr[2][b] - Fr[2][a] * Fr[1][b];
                Cr[1][c] = Fr[2][a] * Fr[0][b] - Fr[0][a] * Fr[2][b];
                Cr[2][c] = Fr[0][a] * Fr[1][b] - Fr[1][a] * Fr[0][b];
            }
            R Pm[3][3];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 3; ++c) Pm[r][c] = (R)mu * Fr[r][c] + s * Cr[r][c];
            R G[3][3];  // h^2 V P B^T: column j -> gradient of vertex j+1
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    R acc = 0;
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc += Pm[r][c] * (R)B[j][c];
                    G[r][j] = (R)h2V * acc;
                }
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                atomicAdd(&g[3 * vid[0] + r], -(G[r][0] + G[r][1] + G[r][2]));
#pragma unroll
                for (int j = 0; j < 3; ++j) atomicAdd(&g[3 * vid[j + 1] + r], G[r][j]);
            }
        }
    }
    warp_add_to(E, e);
}

template <class R>
__global__ void k_barrier(Dev<R> D, ContactBuf C, R* __restrict__ g, double* E) {
    int n = min(*C.count, D.cap);
    double e = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double b, b1, b2;
        barrier3(C.d[i], D.dhat, b, b1, b2);
        e += D.kappa * b;
        if (g) {
            int4 q = C.v[i];
            int vid[4] = {q.x, q.y, q.z, q.w};
            double bp = C.bp[i];
            double r0 = C.r[3 * i], r1 = C.r[3 * i + 1], r2 = C.r[3 * i + 2];
            int nvv = C.type[i] == 2 ? 1 : 4;
            for (int j = 0; j < nvv; ++j) {
                double s = bp * C.w[4 * i + j];
                atomicAdd(&g[3 * vid[j]], (R)(s * r0));
                atomicAdd(&g[3 * vid[j] + 1], (R)(s * r1));
                atomicAdd(&g[3 * vid[j] + 2], (R)(s * r2));
            }
        }
    }
    warp_add_to(E, e);
}

template <class R>
__global__ void k_accept(Dev<R> D) {
    Scalars* S = D.S;
    double Et = S->E_try;
    const double Ek = S->E_k;
    // E(x_try) <= E(x_k) up to the rounding of the two computed energies
    S->accepted = (Et <= Ek + (D.tau_rel * fabs(Ek) + D.tau_abs)) ? 1 : 0;
    if (S->accepted) S->E_k = Et;
}

template <class R>
__global__ void k_zero_scalars(Dev<R> D) {
    Scalars* S = D.S;
    S->gz = S->gp = S->gzprev = 0.0;
    S->zHz = S->zHp = S->pHp = 0.0;
    S->znorm = 0.0;
    S->pmax = 0.0;
    S->maxdisp = 0.0;
}

// ---- scan: block sums, scan of sums, block scan + offset
__global__ void k_scan_sums(const int* in, int n, int* sums) {
    __shared__ int sh[32];
    int i = blockIdx.x * 1024 + threadIdx.x;
    int v = i < n ? in[i] : 0;
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        int w = sh[threadIdx.x];
        w = warp_sum(w);
        if (threadIdx.x == 0) sums[blockIdx.x] = w;
    }
}

__global__ void k_scan_top(int* sums, int nb) {
    // single block, sequential over chunks of 1024
    __shared__ int sh[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < nb ? sums[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) sums[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += sh[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void k_scan_apply(const int* in, int* out, int n, const int* sums) {
    __shared__ int sh[1024];
    int i = blockIdx.x * 1024 + threadIdx.x;
    int v = i < n ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sums[blockIdx.x] + sh[threadIdx.x] - v;
    if (i == n - 1) out[n] = sums[blockIdx.x] + sh[threadIdx.x];
}

}  // namespace

void scan_exclusive(const int* in, int* out, int n, int* tmp, cudaStream_t st) {
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(int), st);
        return;
    }
    int nb = (n + 1023) / 1024;
    KL(k_scan_sums<<<nb, 1024, 0, st>>>(in, n, tmp));
    KL(k_scan_top<<<1, 1024, 0, st>>>(tmp, nb));
    KL(k_scan_apply<<<nb, 1024, 0, st>>>(in, out, n, tmp));
}

template <class R>
void launch_predict(const Dev<R>& D, cudaStream_t st) {
    KL(k_predict<R><<<nblk(3LL * D.nv), kT, 0, st>>>(D));
}

template <class R>
void launch_trial_positions(const Dev<R>& D, int mode, double c, cudaStream_t st) {
    KL(k_trial<R><<<nblk(3LL * D.nv), kT, 0, st>>>(D, mode, c));
}

template <class R>
void launch_energy_grad(const Dev<R>& D, const double* x, const ContactBuf& C, R* g, double* E, cudaStream_t st) {
    cudaMemsetAsync(E, 0, sizeof(double), st);
    KL(k_inertia<R><<<nblk(D.nv), kT, 0, st>>>(D, x, g, E));
    if constexpr (sizeof(R) == 4)
        KL(k_elastic_df<<<nblk(D.nt), kT, 0, st>>>(D, g, E));
    else
        KL(k_elastic<R><<<nblk(D.nt), kT, 0, st>>>(D, x, g, E));
    KL(k_barrier<R><<<1184, kT, 0, st>>>(D, C, g, E));
}

template <class R>
void launch_accept(const Dev<R>& D, cudaStream_t st) {
    KL(k_accept<R><<<1, 1, 0, st>>>(D));
}

template <class R>
void launch_zero_scalars(const Dev<R>& D, cudaStream_t st) {
    KL(k_zero_scalars<R><<<1, 1, 0, st>>>(D));
}

#define INST(R)                                                                                              \
    template void launch_predict<R>(const Dev<R>&, cudaStream_t);                                            \
    template void launch_trial_positions<R>(const Dev<R>&, int, double, cudaStream_t);                       \
    template void launch_energy_grad<R>(const Dev<R>&, const double*, const ContactBuf&, R*, double*,        \
                                        cudaStream_t);                                                       \
    template void launch_accept<R>(const Dev<R>&, cudaStream_t);                                             \
    template void launch_zero_scalars<R>(const Dev<R>&, cudaStream_t);
INST(double)
INST(float)
#undef INST

}  // namespace ipcb
