/* Oracle: stable neo-Hookean tet elasticity (the h^2 Psi term of Eq. 1).
 * Test infrastructure only.
 *
 * Reading (the paper cites Smith et al. 2018 without a formula): the
 * rest-stable SNH energy density
 *     Psi(F) = mu/2 (tr(F^T F) - 3) - mu (J - 1) + lambda/2 (J - 1)^2,
 * J = det F, which is Smith et al.'s simplified form up to a constant.  Its
 * first Piola stress is P = mu F + (lambda (J - 1) - mu) cof(F) and
 *     dP/dF = mu I + lambda vec(cof F) vec(cof F)^T + (lambda (J-1) - mu) d cof/dF.
 * The Hessian used for H_base is the PSD projection of dP/dF (eigenvalues
 * clamped at zero), i.e. the projected Newton Hessian of IPC.
 *
 * Conventions: 3x3 matrices are row-major M[r*3+c]; vec(F) is column-major,
 * vec[3c + r] = F[r][c] (columns f_c of F are contiguous).
 * F = Ds Dm^-1 with Ds = [x1 - x0, x2 - x0, x3 - x0].
 */
#include "o_internal.h"

static double det3(const double* M) {
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}

/* cofactor matrix columns: cof = [f1 x f2, f2 x f0, f0 x f1] */
static void cofactor(const double* F, double* C) {
    double f[3][3];
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) f[c][r] = F[r * 3 + c];
    for (int c = 0; c < 3; ++c) {
        const double* a = f[(c + 1) % 3];
        const double* b = f[(c + 2) % 3];
        double x[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
        for (int r = 0; r < 3; ++r) C[r * 3 + c] = x[r];
    }
}

double o_snh_psi(const double* F, double mu, double lam) {
    double Ic = 0.0;
    for (int i = 0; i < 9; ++i) Ic += F[i] * F[i];
    double J = det3(F);
    return 0.5 * mu * (Ic - 3.0) - mu * (J - 1.0) + 0.5 * lam * (J - 1.0) * (J - 1.0);
}

static void snh_P(const double* F, double mu, double lam, double* P) {
    double C[9];
    cofactor(F, C);
    double J = det3(F);
    for (int i = 0; i < 9; ++i) P[i] = mu * F[i] + (lam * (J - 1.0) - mu) * C[i];
}

/* hat(a) b = a x b, written into the 3x3 block at (rb, cb) of a 9x9 with
 * scale s */
static void add_hat(double* H, int rb, int cb, const double* a, double s) {
    double h[9] = {0, -a[2], a[1], a[2], 0, -a[0], -a[1], a[0], 0};
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) H[(rb * 3 + r) * 9 + cb * 3 + c] += s * h[r * 3 + c];
}

void o_snh_dPdF(const double* F, double mu, double lam, double* H) {
    double f[3][3];
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) f[c][r] = F[r * 3 + c];
    double C[9];
    cofactor(F, C);
    double g[9];
    for (int c = 0; c < 3; ++c)
        for (int r = 0; r < 3; ++r) g[3 * c + r] = C[r * 3 + c];
    double J = det3(F);
    double s = lam * (J - 1.0) - mu;
    for (int i = 0; i < 81; ++i) H[i] = 0.0;
    for (int i = 0; i < 9; ++i) H[i * 9 + i] = mu;
    for (int i = 0; i < 9; ++i)
        for (int j = 0; j < 9; ++j) H[i * 9 + j] += lam * g[i] * g[j];
    /* d cof_c / d f_c' blocks */
    add_hat(H, 0, 1, f[2], -s);
    add_hat(H, 0, 2, f[1], s);
    add_hat(H, 1, 0, f[2], s);
    add_hat(H, 1, 2, f[0], -s);
    add_hat(H, 2, 0, f[1], -s);
    add_hat(H, 2, 1, f[0], s);
}

/* V*Psi, its gradient over the 4 vertices and V * G^T dPdF G (projected if
 * asked), where G maps the 12 vertex coordinates to vec(F). */
void o_snh_tet(const double* B, double vol, double mu, double lam, const double* x12, double* e,
               double* g12, double* H144, int project) {
    double Ds[9], F[9];
    for (int j = 0; j < 3; ++j)
        for (int r = 0; r < 3; ++r) Ds[r * 3 + j] = x12[3 * (j + 1) + r] - x12[r];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double t = 0.0;
            for (int j = 0; j < 3; ++j) t += Ds[r * 3 + j] * B[j * 3 + c];
            F[r * 3 + c] = t;
        }
    if (e) *e = vol * o_snh_psi(F, mu, lam);
    if (g12) {
        double P[9], PBt[9];
        snh_P(F, mu, lam, P);
        for (int r = 0; r < 3; ++r)
            for (int j = 0; j < 3; ++j) {
                double t = 0.0;
                for (int c = 0; c < 3; ++c) t += P[r * 3 + c] * B[j * 3 + c];
                PBt[r * 3 + j] = vol * t;
            }
        for (int r = 0; r < 3; ++r) {
            g12[r] = -(PBt[r * 3 + 0] + PBt[r * 3 + 1] + PBt[r * 3 + 2]);
            for (int j = 0; j < 3; ++j) g12[3 * (j + 1) + r] = PBt[r * 3 + j];
        }
    }
    if (H144) {
        double D[81];
        o_snh_dPdF(F, mu, lam, D);
        if (project) o_psd_project(9, D);
        /* G: 9 x 12 */
        double G[9 * 12];
        memset(G, 0, sizeof G);
        for (int c = 0; c < 3; ++c)
            for (int r = 0; r < 3; ++r) {
                int row = 3 * c + r;
                double sum = 0.0;
                for (int j = 0; j < 3; ++j) {
                    G[row * 12 + 3 * (j + 1) + r] = B[j * 3 + c];
                    sum += B[j * 3 + c];
                }
                G[row * 12 + r] = -sum;
            }
        double DG[9 * 12];
        for (int i = 0; i < 9; ++i)
            for (int k = 0; k < 12; ++k) {
                double t = 0.0;
                for (int j = 0; j < 9; ++j) t += D[i * 9 + j] * G[j * 12 + k];
                DG[i * 12 + k] = t;
            }
        for (int a = 0; a < 12; ++a)
            for (int b = 0; b < 12; ++b) {
                double t = 0.0;
                for (int i = 0; i < 9; ++i) t += G[i * 12 + a] * DG[i * 12 + b];
                H144[a * 12 + b] = vol * t;
            }
    }
}

void o_tet_gather(const OScene* s, int t, const double* x, double* x12) {
    for (int j = 0; j < 4; ++j)
        for (int r = 0; r < 3; ++r) x12[3 * j + r] = x[3 * s->tets[4 * t + j] + r];
}
